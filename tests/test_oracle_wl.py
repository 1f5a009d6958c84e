"""Pins of the oracle's widely-linear equaliser (taps on x and conj(x), the
augmented window [x, conj(x)]): the FIR against the real-valued 4-input
butterfly written out, the reduction to the linear FIR when the conjugate
taps are zero, the exact inverse of a transmitter IQ imbalance, and the
recursion removing an imbalance that the linear equaliser cannot."""
import numpy as np
import pytest

from oracle import chain, oracle_format


def _rand(ns, seed):
    r = np.random.default_rng(seed)
    return (r.standard_normal((2, ns)) + 1j * r.standard_normal((2, ns))) * 0.7


def test_wl_fir_equals_the_real_valued_butterfly():
    """Re y = sum (h_r + g_r) a + (h_i - g_i) b, Im y = sum (h_r - g_r) b -
    (h_i + g_i) a with x = a + jb, h, g the taps on x and conj(x)."""
    T, n = 7, 40
    D = (T - 1) // 2
    x = _rand(2 * n + 20, 1)
    r = np.random.default_rng(2)
    hw = r.standard_normal((2, 2, 2 * T)) + 1j * r.standard_normal((2, 2, 2 * T))
    y = chain.fir(x, hw, 3, 3 + n)
    a, b = x.real, x.imag
    want = np.zeros((2, n), dtype=np.complex128)
    for q in range(2):
        for kk in range(n):
            k = 3 + kk
            re = im = 0.0
            for p in range(2):
                for t in range(T):
                    i = 2 * k + D - t
                    if not 0 <= i < x.shape[1]:
                        continue
                    hr, hi = hw[q, p, t].real, hw[q, p, t].imag
                    gr, gi = hw[q, p, T + t].real, hw[q, p, T + t].imag
                    re += (hr + gr) * a[p, i] + (hi - gi) * b[p, i]
                    im += (hr - gr) * b[p, i] - (hi + gi) * a[p, i]
            want[q, kk] = re + 1j * im
    assert np.max(np.abs(y - want)) < 1e-12


def test_wl_fir_with_zero_conjugate_taps_is_the_linear_fir():
    T = 15
    x = _rand(300, 3)
    r = np.random.default_rng(4)
    h = r.standard_normal((2, 2, T)) + 1j * r.standard_normal((2, 2, T))
    hw = np.concatenate([h, np.zeros_like(h)], axis=2)
    assert np.array_equal(chain.fir(x, hw, 10, 100), chain.fir(x, h, 10, 100))
    assert np.array_equal(chain.center_spike(T, True)[:, :, :T], chain.center_spike(T))


def _iq_imbalanced(n, alpha, beta, seed):
    """Noiseless QPSK per polarisation at 2 samples per symbol (even samples
    carry the symbol), with the imbalance x = alpha s + beta conj(s)."""
    fmt = oracle_format("dp_qpsk")
    r = np.random.default_rng(seed)
    s = fmt.points[r.integers(0, 4, size=(2, n))]
    x = np.zeros((2, 2 * n), dtype=np.complex128)
    x[:, 0::2] = alpha * s + beta * np.conj(s)
    return fmt, s, x


def test_wl_taps_invert_an_iq_imbalance_exactly():
    """h = alpha / Delta, g = -conj(beta) / Delta at the centre tap with
    Delta = |alpha|^2 - |beta|^2 give y = s exactly."""
    alpha, beta = 1.0 * np.exp(0.05j), 0.2 * np.exp(0.7j)
    fmt, s, x = _iq_imbalanced(200, alpha, beta, 5)
    T = 7
    D = (T - 1) // 2
    delta = abs(alpha) ** 2 - abs(beta) ** 2
    hw = np.zeros((2, 2, 2 * T), dtype=np.complex128)
    for q in range(2):
        hw[q, q, D] = alpha / delta
        hw[q, q, T + D] = -np.conj(beta) / delta
    y = chain.fir(x, hw, 0, 200)
    assert np.max(np.abs(y - s)) < 1e-12


def test_wl_dd_lms_removes_an_imbalance_the_linear_one_cannot():
    """DD-LMS from the identity on the imbalanced noiseless stream: the
    widely-linear error energy falls to near zero, the linear one stays at
    the floor |beta|^2 of the conjugate term."""
    alpha, beta = 1.0, 0.25 * np.exp(0.4j)
    fmt, s, x = _iq_imbalanced(6000, alpha, beta, 6)
    T = 7
    p = chain.RxParams(taps=T, n_cma=0, mu=5e-3)
    ks = range(10, 5900)
    phase = {k: 0.0 for k in ks}
    out = {}
    for wl in (False, True):
        h = chain.lms(x, chain.center_spike(T, wl), ks, fmt, p, phase=phase)
        y = chain.fir(x, h, 5000, 5900)
        out[wl] = np.mean(np.abs(y - s[:, 5000:5900]) ** 2)
    assert out[True] < 1e-6
    assert out[False] > 0.5 * abs(beta) ** 2


def test_wl_chain_on_an_iq_imbalanced_stream():
    """The whole oracle chain on DP-16QAM (18 dB) with a transmitter IQ
    imbalance (15 %, 0.12 rad): the linear butterfly leaves an error floor
    that the widely-linear one removes."""
    from paper_2108_07004_gb300 import synth
    n = 1 << 13
    st = synth.make_stream("dp_16qam", n, seed=synth.stream_seed(13, 9), esn0_db=18.0, cd_ps_per_nm=1360.0,
                           linewidth_ts=1e-5, iq_imbalance=(0.15, 0.12))
    fmt = oracle_format("dp_16qam")
    base = dict(cd_ps_per_nm=1360.0, n_fft=1024, n_ov=256, taps=15, bps_phases=32, block=2048, n_pre=2048)
    lin = chain.run_chain(st.rx, fmt, chain.RxParams(**base), ref_bits=st.bits)
    wl = chain.run_chain(st.rx, fmt, chain.RxParams(**base, widely_linear=True), ref_bits=st.bits)
    assert wl.stats["bit_errors"] * 3 < lin.stats["bit_errors"], (wl.stats["bit_errors"], lin.stats["bit_errors"])
