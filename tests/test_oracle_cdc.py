"""Pins of the oracle's CD compensation (A1) against physics and brute force."""
import numpy as np
import pytest

from oracle import chain
from paper_2108_07004_gb300 import synth


def test_numpy_fft_matches_naive_dft():
    # the oracle uses numpy's FFT as a step; check it against the DFT sum
    rng = np.random.default_rng(1)
    for n in (8, 64, 256):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        k = np.arange(n)
        naive = np.array([np.sum(x * np.exp(-2j * np.pi * kk * k / n)) for kk in k])
        assert np.max(np.abs(np.fft.fft(x) - naive)) < 1e-10 * n
        assert np.max(np.abs(np.fft.ifft(np.fft.fft(x)) - x)) < 1e-12


@pytest.mark.parametrize("f0", [-10e9, 6e9])
def test_cd_group_delay_matches_dispersion_physics(f0):
    """A pulse centred at frequency offset f0 through H_CD arrives shifted by
    D*L*dlambda with dlambda = -lambda^2 f0 / c (D = d tau / d lambda)."""
    fs, n, cd = 56e9, 1 << 14, 17000.0
    t = (np.arange(n) - n // 2) / fs
    pulse = np.exp(-t ** 2 / (2 * (150e-12) ** 2)) * np.exp(2j * np.pi * f0 * t)
    f = np.fft.fftfreq(n, 1 / fs)
    out = np.fft.ifft(np.fft.fft(pulse) * chain.cd_response(f, cd, 1550e-9))
    w_in, w_out = np.abs(pulse) ** 2, np.abs(out) ** 2
    shift = np.sum(t * w_out) / np.sum(w_out) - np.sum(t * w_in) / np.sum(w_in)
    dlam_nm = -(1550e-9) ** 2 * f0 / chain.C_LIGHT * 1e9
    expect = cd * dlam_nm * 1e-12                    # ps/nm * nm -> s
    assert abs(shift - expect) < 1e-3 * abs(expect)


def test_overlap_save_equals_linear_convolution_for_short_filter():
    """With an impulse response confined to +-n_ov/2, overlap-save with the
    symmetric discard is exactly the linear (centred) convolution."""
    rng = np.random.default_rng(2)
    p = chain.RxParams(n_fft=256, n_ov=64)
    half = p.n_ov // 2
    g = rng.standard_normal(p.n_ov + 1) + 1j * rng.standard_normal(p.n_ov + 1)  # taps -half..half
    hcirc = np.zeros(p.n_fft, complex)
    for i, v in enumerate(g):
        hcirc[(i - half) % p.n_fft] = v
    H = np.fft.fft(hcirc)
    r = rng.standard_normal((2, 1000)) + 1j * rng.standard_normal((2, 1000))
    out = chain.cdc(r, p, H)
    for pol in range(2):
        full = np.convolve(r[pol], g)              # index i + half aligns to output i
        ref = full[half: half + r.shape[1]]
        assert np.max(np.abs(out[pol] - ref)) < 1e-11


@pytest.mark.parametrize("cd,nfft,nov", [(1360.0, 1024, 256), (17000.0, 4096, 1024)])
def test_cdc_recovers_symbols_on_noiseless_link(cd, nfft, nov):
    """Noiseless link with CD and RRC shaping: CD inversion plus matched
    filtering returns the transmitted symbols at the even samples."""
    n = 1 << 13
    st = synth.make_stream("dp_qpsk", n, seed=5, esn0_db=99, cd_ps_per_nm=cd,
                           linewidth_ts=0.0, rotation=False, noise=False, phase0=0.0)
    p = chain.RxParams(cd_ps_per_nm=cd, n_fft=nfft, n_ov=nov)
    x = chain.cdc(st.rx.astype(np.complex128), p)
    edge = 512
    err = np.abs(x[:, 2 * edge: 2 * (n - edge): 2] - st.sym[:, edge: n - edge])
    assert np.max(err) < 2e-3
    assert np.sqrt(np.mean(err ** 2)) < 3e-4
    # the wrong sign of the CD exponent does not compensate
    p_bad = chain.RxParams(cd_ps_per_nm=-cd, n_fft=nfft, n_ov=nov)
    xb = chain.cdc(st.rx.astype(np.complex128), p_bad)
    errb = np.abs(xb[:, 2 * edge: 2 * (n - edge): 2] - st.sym[:, edge: n - edge])
    assert np.sqrt(np.mean(errb ** 2)) > 0.1


def test_cdc_unitary_spectrum_parseval():
    """|conj(H_CD)| = 1, so with H_MF = 1 in band the frame energy is kept."""
    f = np.linspace(-28e9, 28e9, 1001)
    h = chain.cd_response(f, 34000.0, 1550e-9)
    assert np.max(np.abs(np.abs(h) - 1)) < 1e-14
    rc = chain.raised_cosine(f, 28e9, 0.1)
    # raised cosine is Nyquist: r(f) + r(f - Rs) = 1 on the transition band
    ff = np.linspace(0.45 * 28e9, 0.55 * 28e9, 101)
    s = chain.raised_cosine(ff, 28e9, 0.1) + chain.raised_cosine(ff - 28e9, 28e9, 0.1)
    assert np.max(np.abs(s - 1)) < 1e-12
    assert rc.max() == 1.0


def test_cdc_without_matched_filter_and_dispersion_is_the_identity():
    """matched_filter = False with no dispersion leaves the multiply at 1:
    overlap-save returns its input exactly (the chain after the KK front-end
    and the static equaliser, which did the matched filtering)."""
    rng = np.random.default_rng(4)
    r = rng.standard_normal((2, 5000)) + 1j * rng.standard_normal((2, 5000))
    for nfft, nov in ((1024, 256), (4096, 1024)):
        p = chain.RxParams(cd_ps_per_nm=0.0, n_fft=nfft, n_ov=nov, matched_filter=False)
        assert np.max(np.abs(chain.cdc(r, p) - r)) < 1e-12
        assert np.max(np.abs(chain.cdc(r, chain.RxParams(cd_ps_per_nm=0.0, n_fft=nfft, n_ov=nov)) - r)) > 0.1
