"""Pins of the oracle's butterfly FIR (A2) and CMA/DD-LMS (A3)."""
import numpy as np
import pytest

from oracle import chain, oracle_format
from paper_2108_07004_gb300 import synth


def _rand(shape, rng):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_fir_center_spike_is_decimation():
    rng = np.random.default_rng(3)
    x = _rand((2, 400), rng)
    y = chain.fir(x, chain.center_spike(15), 0, 200)
    assert np.array_equal(y, x[:, 0::2])


def test_fir_matches_numpy_convolution():
    """sum_t conj(h[t]) x[2k+D-t] is a convolution with conj(h) sampled at
    even outputs, shifted by D."""
    rng = np.random.default_rng(4)
    T, D = 31, 15
    x = _rand((2, 600), rng)
    h = _rand((2, 2, T), rng)
    y = chain.fir(x, h, 0, 300)
    for q in range(2):
        acc = np.zeros(600 + T - 1, complex)
        for pol in range(2):
            acc += np.convolve(x[pol], np.conj(h[q, pol]))
        # full[i] = sum_t conj(h[t]) x[i - t]; we need i = 2k + D
        assert np.max(np.abs(y[q] - acc[D: D + 600: 2])) < 1e-12


def _equalised_link(fmt_name, n, J=True, seed=11):
    st = synth.make_stream(fmt_name, n, seed=seed, esn0_db=99, cd_ps_per_nm=0.0,
                           linewidth_ts=0.0, rotation=J, noise=False, phase0=0.0)
    p = chain.RxParams(n_fft=1024, n_ov=256)
    return st, p, chain.cdc(st.rx.astype(np.complex128), p)


def test_cma_converges_to_inverse_of_known_rotation():
    """Noiseless, CD-free DP-QPSK through a fixed unitary J: after CMA the
    equalised output is the transmitted symbols up to a diagonal or
    anti-diagonal phase matrix, with constant modulus.

    (The T/2-spaced taps are not unique: out of the signal band the
    noiseless input carries no energy, so the check is on the output.)"""
    fmt = oracle_format("dp_qpsk")
    st, p, x = _equalised_link("dp_qpsk", 6000)
    p.mu = 3e-3
    h = chain.center_spike(p.taps)
    for _ in range(2):
        h = chain.lms(x, h, range(6000), fmt, p, force_cma=True)
    y = chain.fir(x, h, 5000, 6000)
    s = st.sym[:, 5000:6000]
    A = (y @ np.conj(s).T) @ np.linalg.inv(s @ np.conj(s).T)    # y ~ A s
    diag = abs(A[0, 0]) ** 2 + abs(A[1, 1]) ** 2
    anti = abs(A[0, 1]) ** 2 + abs(A[1, 0]) ** 2
    big, small = max(diag, anti), min(diag, anti)
    assert small < 1e-3 and abs(big - 2) < 2e-2
    assert np.sqrt(np.mean(np.abs(y - A @ s) ** 2)) < 2e-2
    assert np.var(np.abs(y) ** 2) < 2e-4
    # the identity start (no adaptation) is far from that
    y0 = chain.fir(x, chain.center_spike(p.taps), 5000, 6000)
    assert np.var(np.abs(y0) ** 2) > 1e-2


def test_dd_lms_fixed_point_with_true_decisions():
    """With exact taps, exact phase and noiseless input, every DD error is 0
    (to rounding) and the taps do not move."""
    fmt = oracle_format("gs4d64")
    rng = np.random.default_rng(13)
    n = 1200
    bits = rng.integers(0, 2, size=(n, 6), dtype=np.uint8)
    s = fmt.symbols_from_bits(bits)
    J = synth.haar_unitary(np.random.Generator(np.random.PCG64(5)))
    x = np.zeros((2, 2 * n), complex)
    x[:, 0::2] = J @ s                                  # symbol-instant samples
    x[:, 1::2] = J @ (0.5 * (s + np.roll(s, -1, axis=1)))
    p = chain.RxParams(n_cma=0)
    T, D = p.taps, (p.taps - 1) // 2
    h = np.zeros((2, 2, T), complex)
    h[:, :, D] = np.conj(np.linalg.inv(J))              # y = conj(h) x = J^-1 x
    phase = {k: 0.0 for k in range(100, 1100)}
    info = chain.LmsInfo()
    h2 = chain.lms(x, h, range(100, 1100), fmt, p, phase=phase, info=info)
    assert np.max(np.abs(h2 - h)) < 1e-12
    assert len(info.dd_margin) == 1000 and min(m for _, m in info.dd_margin) > 0.01
    # a wrong phase makes the same recursion move the taps
    h3 = chain.lms(x, h, range(100, 300), fmt, p, phase={k: 0.2 for k in range(100, 300)})
    assert np.max(np.abs(h3 - h)) > 1e-3


def test_dd_lms_converges_from_perturbed_taps():
    fmt = oracle_format("dp_16qam")
    st, p, x = _equalised_link("dp_16qam", 8000, seed=12)
    T, D = p.taps, (p.taps - 1) // 2
    h = np.zeros((2, 2, T), complex)
    h[:, :, D] = np.conj(np.linalg.inv(st.J))
    rng = np.random.default_rng(0)
    h0 = h + 0.02 * _rand(h.shape, rng)
    p.n_cma, p.mu = 0, 2e-3
    phase = {k: 0.0 for k in range(8000)}
    h2 = chain.lms(x, h0, range(7000), fmt, p, phase=phase)
    s_ref = st.sym[:, 7000:8000]
    before = np.mean(np.abs(chain.fir(x, h0, 7000, 8000) - s_ref) ** 2)
    after = np.mean(np.abs(chain.fir(x, h2, 7000, 8000) - s_ref) ** 2)
    assert after < 0.05 * before


def test_training_alignment_fixes_swap_and_phase():
    fmt = oracle_format("dp_qpsk")
    st, p, x = _equalised_link("dp_qpsk", 2000, J=False)
    T, D = p.taps, (p.taps - 1) // 2
    h = np.zeros((2, 2, T), complex)
    # equaliser that swaps the polarisations and rotates them
    h[0, 1, D] = np.exp(-1j * 0.7)      # y0 = conj(h01) x1 = e^{j0.7} x1
    h[1, 0, D] = np.exp(1j * 2.1)       # y1 = e^{-j2.1} x0
    ref = fmt.symbols_from_bits(st.bits[:1000])
    h2 = chain.align_training(x, h, ref)
    y = chain.fir(x, h2, 0, 1000)
    # the first symbols see the stream-start edge of the pulse shaping
    assert np.max(np.abs(y[:, 100:] - ref[:, 100:])) < 2e-3


def test_cma_radius():
    assert abs(oracle_format("dp_qpsk").cma_radius2() - 1.0) < 1e-12
    # 16QAM: E|s|^4 = 1.32 for unit energy
    assert abs(oracle_format("dp_16qam").cma_radius2() - 1.32) < 1e-12


def test_training_stage_recovers_a_singular_cma_solution():
    """CMA can let both outputs capture the same polarisation.  The training
    stage (order/phase from the known symbols, data-aided phase, data-aided
    LMS) recovers both polarisations."""
    fmt = oracle_format("gs4d64")
    st, p, x = _equalised_link("gs4d64", 3000)
    T, D = p.taps, (p.taps - 1) // 2
    Jinv = np.linalg.inv(st.J)
    h = np.zeros((2, 2, T), complex)
    h[0, :, D] = np.conj(Jinv[1])          # both outputs see polarisation Y
    h[1, :, D] = np.conj(Jinv[1]) * np.exp(0.4j)
    ref = fmt.symbols_from_bits(st.bits[:2048])
    y0 = chain.fir(x, h, 0, 2048)
    assert np.mean(np.abs(y0[0] - ref[0]) ** 2) > 0.5
    h = chain.align_training(x, h, ref)
    b, m = chain.train_phase(chain.fir(x, h, 0, 2048), ref, 64, 64, 4)
    phi = chain.phase_of(b, m, 64, 4)
    p.mu = 2e-3
    for _ in range(3):
        h = chain.lms_trained(x, h, range(2048), ref, phi, p)
    y = chain.fir(x, h, 100, 2048)
    err = np.mean(np.abs(y * np.exp(-1j * phi[100:2048]) - ref[:, 100:2048]) ** 2)
    assert err < 2e-2


def test_train_phase_is_exact_on_grid_phases():
    fmt = oracle_format("gs4d64")
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2, size=(500, 6), dtype=np.uint8)
    s = fmt.symbols_from_bits(bits)
    step = 2 * np.pi / 4 / 64
    for nk in (-100, -5, 0, 37, 120):       # beyond +-pi/4: no rotational ambiguity
        b, m = chain.train_phase(s * np.exp(1j * nk * step), s, 64, 64, 4)
        assert np.all(b + 64 * m - 32 == nk)
