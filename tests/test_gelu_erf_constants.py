"""The tensor-core inference kernel evaluates GELU with Abramowitz and
Stegun's rational approximation 7.1.26 of erfc (Handbook of Mathematical
Functions, after Hastings), |error| <= 1.5e-7 on erf.  This reads the
constants as written in csrc/k_mlp_tc.cu and checks, in float64, that
they reproduce that bound on erfc and the resulting bound on GELU(a) =
a Phi(a) (a mistyped coefficient breaks it)."""
import math
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2108_07004_gb300", "csrc", "k_mlp_tc.cu")


def _constants():
    text = open(SRC).read()
    p = float(re.search(r"kAsP = ([0-9.e+-]+)f \* 0\.70710678118654752f", text).group(1))
    a = []
    for i in range(1, 6):
        m = re.search(rf"kAs{i} = 0\.5f \* (-?[0-9.]+)f", text)
        a.append(float(m.group(1)))
    return p, a


def _erfc_as(z, p, a):
    t = 1.0 / (1.0 + p * z)
    poly = t * (a[0] + t * (a[1] + t * (a[2] + t * (a[3] + t * a[4]))))
    return poly * np.exp(-z * z)


def test_erfc_approximation_within_the_handbook_bound():
    p, a = _constants()
    z = np.linspace(0.0, 8.0, 200001)
    ref = np.array([math.erfc(v) for v in z])
    assert np.max(np.abs(_erfc_as(z, p, a) - ref)) <= 1.5e-7


def test_gelu_from_the_approximation():
    p, a = _constants()
    x = np.linspace(-12.0, 12.0, 120001)
    q = 0.5 * _erfc_as(np.abs(x) / math.sqrt(2.0), p, a)
    gelu = x * (0.5 + np.copysign(0.5 - q, x))
    ref = np.array([0.5 * v * math.erfc(-v / math.sqrt(2.0)) for v in x])
    assert np.max(np.abs(gelu - ref) / np.maximum(1.0, np.abs(x))) <= 0.75e-7 + 1e-15
