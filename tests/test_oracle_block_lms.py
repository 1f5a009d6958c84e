"""Pins of the oracle's block LMS (groups of P updates sharing the taps at
the group start): it reduces to the sequential recursion at P = 1, one group
equals the closed form written with array operations, a perfectly equalised
noiseless stream is a fixed point, and the chain runs with it."""
import math

import numpy as np
import pytest

from oracle import chain, oracle_format
from paper_2108_07004_gb300 import synth


def _rand(ns, seed):
    r = np.random.default_rng(seed)
    return (r.standard_normal((2, ns)) + 1j * r.standard_normal((2, ns))) * 0.7


def _taps(T, seed):
    r = np.random.default_rng(seed)
    h = chain.center_spike(T) + 0.05 * (r.standard_normal((2, 2, T)) + 1j * r.standard_normal((2, 2, T)))
    return h


@pytest.mark.parametrize("n_cma", [0, 5, 1000])
def test_block_of_one_is_the_sequential_recursion(n_cma):
    fmt = oracle_format("dp_16qam")
    T = 7
    x = _rand(200, 1)
    h = _taps(T, 2)
    ks = range(10, 60)
    p = chain.RxParams(taps=T, n_cma=n_cma, mu=3e-3)
    phase = {k: 0.1 * k for k in ks}
    a = chain.lms(x, h, ks, fmt, p, phase=phase)
    b = chain.lms_block(x, h, ks, fmt, p, 1, phase=phase)
    assert np.array_equal(a, b)


def test_one_group_equals_the_array_form():
    """CMA over one group of P symbols: Y = conj(H) . X for all windows at
    once, E = (R^2 - |Y|^2) Y, H' = H + mu sum_k conj(E_k) X_k (einsum)."""
    fmt = oracle_format("gs4d64")
    T, P, k0 = 15, 16, 40
    x = _rand(400, 3)
    h = _taps(T, 4)
    p = chain.RxParams(taps=T, n_cma=10 ** 9, mu=2e-3)
    D = (T - 1) // 2
    idx = 2 * np.arange(k0, k0 + P)[:, None] + D - np.arange(T)[None, :]          # [P, T]
    X = np.transpose(x[:, idx], (1, 0, 2))                                          # [P, 2, T]
    Y = np.einsum("qpt,kpt->kq", np.conj(h), X)
    E = (fmt.cma_radius2() - np.abs(Y) ** 2) * Y
    want = h + p.mu * np.einsum("kq,kpt->qpt", np.conj(E), X)
    got = chain.lms_block(x, h, range(k0, k0 + P), fmt, p, P)
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("P", [1, 4, 16])
def test_equalised_noiseless_stream_is_a_fixed_point(P):
    """Even samples carry the symbols, odd ones zero, taps = identity: every
    DD output is its own table point, so every error and update is 0."""
    fmt = oracle_format("dp_qpsk")
    T, n = 7, 96
    r = np.random.default_rng(5)
    lab = r.integers(0, fmt.points.shape[0], size=(2, n))
    s = fmt.points[lab]
    x = np.zeros((2, 2 * n), dtype=np.complex128)
    x[:, 0::2] = s
    h = chain.center_spike(T)
    p = chain.RxParams(taps=T, n_cma=0, mu=1e-2)
    ks = range(4, n - 4)
    got = chain.lms_block(x, h, ks, fmt, p, P, phase={k: 0.0 for k in ks})
    assert np.max(np.abs(got - h)) == 0.0


def test_chain_runs_with_block_updates():
    """The whole chain with groups of 16: BER within a few times the exact
    chain's on a 1000 km 4D-64 stream (the block form trades a little
    convergence speed for parallel updates)."""
    n = 1 << 13
    st = synth.make_stream("gs4d64", n, seed=synth.stream_seed(12, 0), esn0_db=13.0,
                           cd_ps_per_nm=17000.0, linewidth_ts=1e-5)
    fmt = oracle_format("gs4d64")
    base = dict(cd_ps_per_nm=17000.0, n_fft=4096, n_ov=1024, taps=31, bps_phases=64, block=2048,
                n_pre=2048)
    ex = chain.run_chain(st.rx, fmt, chain.RxParams(**base), ref_bits=st.bits)
    bl = chain.run_chain(st.rx, fmt, chain.RxParams(**base, lms_block=16), ref_bits=st.bits)
    assert ex.stats["ber"] < 0.02
    assert bl.stats["ber"] <= 3 * ex.stats["ber"] + 1e-3
    assert len(bl.dd_margin) == len(ex.dd_margin)
