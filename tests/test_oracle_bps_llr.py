"""Pins of the oracle's BPS (A4), unwrap, exact LLRs (A5) and counting (A6)."""
import math

import numpy as np
import pytest
from scipy.special import erfc

from oracle import chain, oracle_format
from paper_2108_07004_gb300 import synth


def _symbols(fmt, n, seed):
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2, size=(n, fmt.m), dtype=np.uint8)
    return bits, fmt.symbols_from_bits(bits)


@pytest.mark.parametrize("name,B", [("dp_qpsk", 32), ("dp_16qam", 32), ("gs4d64", 64)])
@pytest.mark.parametrize("theta", [0.3, -1.2, 2.9])
def test_bps_recovers_injected_constant_phase(name, B, theta):
    """Noiseless equalised symbols rotated by theta: the chosen test phase is
    theta modulo the pi/2 symmetry, to within half a grid step."""
    fmt = oracle_format(name)
    _, s = _symbols(fmt, 400, 1)
    y = s * np.exp(1j * theta)
    p = chain.RxParams(bps_phases=B)
    b, gap, _ = chain.bps(y, 0, 400, 400, p, fmt)
    phi = chain.bps_phases(B, 4)[b]
    q = np.pi / 2
    err = (phi - theta + q / 2) % q - q / 2
    assert np.max(np.abs(err)) <= q / (2 * B) + 1e-12


def test_bps_exact_on_grid_phase():
    fmt = oracle_format("gs4d64")
    _, s = _symbols(fmt, 200, 2)
    B = 64
    grid = chain.bps_phases(B, 4)
    y = s * np.exp(1j * grid[17])
    b, _, chosen = chain.bps(y, 0, 200, 200, chain.RxParams(bps_phases=B), fmt)
    assert np.all(b == 17)
    assert np.max(chosen) < 1e-20


def test_bps_window_cost_brute_force():
    """Tiny input: window costs and the argmin by explicit loops."""
    fmt = oracle_format("dp_16qam")
    rng = np.random.default_rng(3)
    _, s = _symbols(fmt, 50, 3)
    y = s * np.exp(0.2j) + 0.15 * (rng.standard_normal(s.shape) + 1j * rng.standard_normal(s.shape))
    p = chain.RxParams(bps_phases=8, bps_window=10)
    a, e, nv = 5, 45, 50
    b, _, _ = chain.bps(y, a, e, nv, p, fmt)
    phis = chain.bps_phases(8, 4)
    for idx, k in enumerate(range(a, e)):
        costs = []
        for ph in phis:
            c = 0.0
            for i in range(k - 5, k + 5):
                if 0 <= i < nv:
                    for pol in range(2):
                        c += min(abs(y[pol, i] * np.exp(-1j * ph) - pt) ** 2 for pt in fmt.points)
            costs.append(c)
        best = min(range(8), key=lambda j: (costs[j], j))
        assert b[idx] == best


def test_unwrap_integer_form_matches_float_definition():
    rng = np.random.default_rng(4)
    B, q = 64, np.pi / 2
    b = rng.integers(0, B, size=2000)
    # avoid exact half-way differences for the float comparison
    b = np.where(np.abs(np.diff(np.concatenate([[B // 2], b]))) == B // 2, (b + 1) % B, b)
    m, _, _ = chain.unwrap(b, 0, B // 2, B)
    phi = (b / B - 0.5) * q
    prev = 0.0
    for k in range(len(b)):
        ph = phi[k] + q * np.floor((prev - phi[k]) / q + 0.5)
        assert abs(ph - (phi[k] + q * m[k])) < 1e-9
        prev = ph


def test_unwrap_tie_rounds_up_and_tracks_slow_drift():
    B = 64
    m, mp, bp = chain.unwrap(np.array([0]), 0, 32, B)   # difference exactly B/2
    assert m[0] == 1 and mp == 1 and bp == 0
    # a phase ramp through several quadrants is followed without slips
    true = np.linspace(0, 3 * np.pi, 3000)
    grid = chain.bps_phases(B, 4)
    b = np.array([np.argmin(np.abs((grid - t + np.pi / 4) % (np.pi / 2) - np.pi / 4)) for t in true])
    m, _, _ = chain.unwrap(b, 0, B // 2, B)
    phi = chain.phase_of(b, m, B, 4)
    assert np.max(np.abs(phi - true)) <= np.pi / (2 * B) + 1e-9


def test_bps_tracks_wiener_phase_noise():
    """Equalised DP-QPSK with Wiener phase noise: the unwrapped estimate
    follows the true phase (RMS error well inside the pi/4 slip limit)."""
    fmt = oracle_format("dp_qpsk")
    n = 6000
    rng = np.random.default_rng(5)
    bits, s = _symbols(fmt, n, 5)
    theta = np.cumsum(rng.standard_normal(n) * np.sqrt(2 * np.pi * 1e-4))
    y = s * np.exp(1j * theta) + 0.1 * (rng.standard_normal(s.shape) + 1j * rng.standard_normal(s.shape))
    p = chain.RxParams(bps_phases=32, bps_window=64)
    b, _, _ = chain.bps(y, 0, n, n, p, fmt)
    m, _, _ = chain.unwrap(b, 0, 16, 32)
    phi = chain.phase_of(b, m, 32, 4)
    off = np.round((theta[0] - phi[0]) / (np.pi / 2)) * np.pi / 2
    assert np.sqrt(np.mean((phi + off - theta) ** 2)) < 0.08


def test_llr_qpsk_closed_form():
    """Gray QPSK per polarisation: LLR = 2 sqrt(2) Re z / sigma^2 (and Im)."""
    fmt = oracle_format("dp_qpsk")
    rng = np.random.default_rng(6)
    z = rng.standard_normal((2, 300)) + 1j * rng.standard_normal((2, 300))
    s2 = 0.37
    L = chain.llr(z, s2, fmt)
    k = 2 * np.sqrt(2) / s2
    ref = np.stack([k * z[0].real, k * z[0].imag, k * z[1].real, k * z[1].imag], axis=1)
    assert np.max(np.abs(L - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", ["dp_qpsk", "dp_16qam", "gs4d64"])
def test_llr_matches_naive_long_double_sum(name):
    """Unshifted sum of exponentials in extended precision on small inputs."""
    fmt = oracle_format(name)
    rng = np.random.default_rng(7)
    _, s = _symbols(fmt, 64, 7)
    z = s + 0.3 * (rng.standard_normal(s.shape) + 1j * rng.standard_normal(s.shape))
    s2 = 0.2
    L = chain.llr(z, s2, fmt)
    bt = fmt.bit_table()
    ld = np.longdouble
    for k in range(z.shape[1]):
        row = []
        groups = [(None, fmt.points)] if fmt.dims == 4 else [(0, fmt.points), (1, fmt.points)]
        for pol, pts in groups:
            if pol is None:
                d = [ld(abs(z[0, k] - pt[0]) ** 2 + abs(z[1, k] - pt[1]) ** 2) for pt in pts]
            else:
                d = [ld(abs(z[pol, k] - pt) ** 2) for pt in pts]
            for i in range(bt.shape[1]):
                s0 = sum(np.exp(-d[j] / ld(s2)) for j in range(len(pts)) if bt[j, i] == 0)
                s1 = sum(np.exp(-d[j] / ld(s2)) for j in range(len(pts)) if bt[j, i] == 1)
                row.append(float(np.log(s0) - np.log(s1)))
        assert np.max(np.abs(L[k] - np.array(row))) < 1e-11 * max(1.0, np.max(np.abs(row)))


def test_gmi_qpsk_equals_bpsk_mutual_information():
    """Gray QPSK in AWGN with exact LLRs: the GMI is 4 x the BPSK mutual
    information at the per-dimension SNR (computed by Gauss-Hermite
    quadrature), within Monte-Carlo error."""
    fmt = oracle_format("dp_qpsk")
    n0 = 10 ** (-6 / 10)
    n = 1 << 17
    rng = np.random.default_rng(8)
    bits, s = _symbols(fmt, n, 8)
    z = s + np.sqrt(n0 / 2) * (rng.standard_normal(s.shape) + 1j * rng.standard_normal(s.shape))
    c = chain.count(chain.llr(z, n0, fmt), bits.astype(float))
    # BPSK +-a with noise var sn2 per real dimension
    a, sn2 = 1 / np.sqrt(2), n0 / 2
    xg, wg = np.polynomial.hermite.hermgauss(80)
    nn = np.sqrt(2 * sn2) * xg
    llr_b = 2 * a * (a + nn) / sn2
    mi = 1 - np.sum(wg * np.logaddexp(0, -llr_b)) / np.sqrt(np.pi) / np.log(2)
    assert abs(c["gmi"] - 4 * mi) < 4e-3


def test_ber_qpsk_awgn_matches_theory():
    fmt = oracle_format("dp_qpsk")
    esn0 = 7.0
    n0 = 10 ** (-esn0 / 10)
    n = 1 << 17
    rng = np.random.default_rng(9)
    bits, s = _symbols(fmt, n, 9)
    z = s + np.sqrt(n0 / 2) * (rng.standard_normal(s.shape) + 1j * rng.standard_normal(s.shape))
    c = chain.count(chain.llr(z, n0, fmt), bits.astype(float))
    pb = 0.5 * erfc(math.sqrt(10 ** (esn0 / 10) / 2))
    sd = math.sqrt(pb * (1 - pb) / c["n_bits"])
    assert abs(c["ber"] - pb) < 4 * sd


def test_sigma2_estimate_close_to_true_noise_at_high_snr():
    fmt = oracle_format("dp_16qam")
    n0 = 10 ** (-20 / 10)
    rng = np.random.default_rng(10)
    _, s = _symbols(fmt, 20000, 10)
    z = s + np.sqrt(n0 / 2) * (rng.standard_normal(s.shape) + 1j * rng.standard_normal(s.shape))
    assert abs(chain.estimate_sigma2(z, fmt) / n0 - 1) < 0.03


def test_quadrant_anchor_recovers_training_quadrant():
    """Blind phase indices that agree with the training phase up to a whole
    number of quadrants (plus a garbled start) are anchored to the training
    quadrant: the anchored unwrap equals the training phase modulo 2 pi."""
    B, S = 64, 4
    rng = np.random.default_rng(11)
    n = 1024
    true_n = np.cumsum(rng.integers(-1, 2, size=n)) + 40          # grid units, drifting
    mt = np.floor_divide(true_n + B // 2, B)
    bt = true_n + B // 2 - mt * B
    for shift in range(4):
        blind = (true_n + shift * B + B // 2) % B                 # b is blind to quadrants
        b = blind.copy()
        b[:60] = rng.integers(0, B, size=60)                       # garbled stream start
        q = chain.quadrant_anchor(b, bt, mt, B, S)
        m, _, _ = chain.unwrap(b, q, B // 2, B)
        nb = b - B // 2 + m * B
        agree = ((nb - true_n) % (S * B)) == 0
        assert agree[100:].mean() > 0.99
