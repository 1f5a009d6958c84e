"""Pins of the static frequency-domain equaliser oracle (Sec. 2: a 203-tap
static equaliser trained offline on a known sequence, applied by an FFT pair
that also resamples from 4 to 2 samples per symbol)."""
import numpy as np

from oracle import fde, kk
from paper_2108_07004_gb300 import synth


def test_training_is_least_squares():
    """With delta = 0 the taps are the library least-squares solution of
    the symbol-instant equations, the regressor matrix built here by brute
    force."""
    rng = np.random.default_rng(1)
    T, K, sps = 21, 400, 4
    x = rng.standard_normal(sps * K + 50) + 1j * rng.standard_normal(sps * K + 50)
    d = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    D = (T - 1) // 2
    U = np.zeros((K, T), dtype=complex)
    for i in range(K):
        for t in range(T):
            n = sps * i + D - t
            if 0 <= n < x.shape[0]:
                U[i, t] = x[n]
    h_ls = np.linalg.lstsq(U, d, rcond=None)[0]
    h = fde.train(x, d, T=T, sps=sps, delta=0.0)
    assert np.max(np.abs(h - h_ls)) < 1e-10 * np.max(np.abs(h_ls))


def test_training_inverts_a_short_pulse_exactly():
    """Noiseless x = sum_i d_i g[n - 4i] with a short pulse g: some taps make
    the symbol instants reproduce d exactly, so the trained equaliser does,
    to the small bias of the regularisation."""
    rng = np.random.default_rng(2)
    K = 3000
    d = (rng.integers(0, 2, K) * 2 - 1) + 1j * (rng.integers(0, 2, K) * 2 - 1)
    g = np.array([0.1, 0.3, 0.6, 1.0, 0.5, 0.2, -0.1])
    u = np.zeros(4 * K, dtype=complex)
    u[::4] = d
    x = np.convolve(u, g)[3:3 + 4 * K]              # pulse centred on the symbol instant
    h = fde.train(x, d[:2000], T=203, delta=1e-12)
    U = fde.regressors(x, K, 203)
    r = U @ h - d
    sl = slice(100, K - 100)
    assert np.mean(np.abs(r[sl]) ** 2) < 1e-8


def test_apply_resamples_in_band_tones_exactly():
    """Tones on multiples of fs/1024 are periodic in every frame (away from
    the stream ends, where the frames are zero-padded): with the
    identity equaliser (h[D] = 1) the output is x[2m] for in-band tones and
    0 for a tone outside |f| < fs/4; with any taps an in-band tone k0 comes
    out multiplied by sum_t h[t] e^{-j 2 pi k0 (t - D) / 1024}."""
    n = 8 * 1024
    t_ = np.arange(n)
    ks = (3, -100, 200, -255)
    x = sum(np.exp(2j * np.pi * k * t_ / 1024) * (1 + 0.1 * i) for i, k in enumerate(ks))
    hid = np.zeros(203, dtype=complex)
    hid[101] = 1.0
    sl = slice(512, -512)                      # frames away from the zero-padded ends
    for n_ov in (256, 512):
        y = fde.apply(x, hid, n_ov=n_ov)
        assert np.max(np.abs(y[sl] - x[0::2][sl])) < 1e-11
    y = fde.apply(np.exp(2j * np.pi * 300 * t_ / 1024), hid)
    assert np.max(np.abs(y[sl])) < 1e-12
    rng = np.random.default_rng(3)
    h = rng.standard_normal(203) + 1j * rng.standard_normal(203)
    k0 = 37
    x0 = np.exp(2j * np.pi * k0 * t_ / 1024)
    gain = np.sum(h * np.exp(-2j * np.pi * k0 * (np.arange(203) - 101) / 1024))
    y = fde.apply(x0, h)
    assert np.max(np.abs(y[sl] - gain * x0[0::2][sl])) < 1e-10 * abs(gain)


def test_trained_equaliser_after_kk_front_end():
    """The paper's receiver order: KK field -> trained static equaliser with
    resampling.  On a 16QAM KK signal (14 dB CSPR, Es/N0 25 dB) the
    symbol-instant EVM falls below -20 dB and beats the untrained identity
    (with its best complex gain) by more than 1.5 dB."""
    k = synth.make_kk_stream("dp_16qam", 16384, seed=3, cspr_db=14.0, esn0_db=25.0)
    x = kk.kk_field_from_codes(k.codes, scale=k.scale, dc=k.dc, fc_step=k.fc_step, floor=1e-3)
    h = fde.train(x, k.sym[:4096])
    ys = fde.apply(x, h)[0::2]
    sl = slice(100, -100)
    p = np.mean(np.abs(k.sym) ** 2)
    evm = 10 * np.log10(np.mean(np.abs(ys[sl] - k.sym[sl]) ** 2) / p)
    hid = np.zeros(203, dtype=complex)
    hid[101] = 1.0
    y0 = fde.apply(x, hid)[0::2]
    g = np.vdot(y0, k.sym) / np.vdot(y0, y0)
    evm0 = 10 * np.log10(np.mean(np.abs(g * y0[sl] - k.sym[sl]) ** 2) / p)
    assert evm < -20.0 and evm < evm0 - 1.5
