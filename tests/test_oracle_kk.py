"""Pins of the Kramers-Kronig front-end oracle (Sec. 2: square root and
logarithm of the detected intensity, frequency-domain Hilbert transform by
an overlap-save FFT pair, field reconstruction, downconversion)."""
import numpy as np
import pytest

from oracle import kk
from paper_2108_07004_gb300 import synth


def test_frame_phase_is_minus_scipy_hilbert():
    """The spectral step equals the library's analytic-signal construction:
    scipy.signal.hilbert(l) = l + j H{l}; the phase of a field with its
    signal below the carrier is -H{ln|E|}."""
    ss = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    for n in (256, 1024):
        l = rng.standard_normal(n)
        phi, lbar = kk.frame_phase(l)
        assert np.max(np.abs(phi + np.imag(ss.hilbert(l)))) < 1e-12
        assert abs(lbar - l.mean()) < 1e-14


@pytest.mark.parametrize("n_ov", [256, 512])
def test_single_tone_minimum_phase_field_is_exact(n_ov):
    """E = A + b e^{-j w n} with b < A is minimum phase; with w a multiple
    of 2 pi / 1024 every frame holds whole periods of ln|E| and its
    harmonics stay below Nyquist, so the reconstruction is exact: the
    output is b e^{-j w n} (fc = 0), the carrier A removed."""
    N = 16384
    n = np.arange(N)
    A, b = 1.3, 0.4
    s = b * np.exp(-2j * np.pi * 2 / 1024 * n)
    I = np.abs(A + s) ** 2
    out = kk.kk_field(I, pad=float(np.mean(I)), fc_step=0, n_ov=n_ov)
    sl = slice(1024, N - 1024)
    assert np.max(np.abs(out[sl] - s[sl])) < 1e-12


def test_downconversion_of_a_tone_below_the_carrier():
    """s = b e^{+j 2 pi 8/1024 n} placed at fc = 132/1024 below the carrier
    (E = A + s e^{-j 2 pi fc n}); the front-end returns s.  b/A = 0.01 keeps
    the aliased fifth harmonic of ln|E| below 1e-10 A."""
    N = 16384
    n = np.arange(N)
    fc_step = 132 << 22                        # 132/1024 cycles per sample
    A, b = 2.0, 0.02
    s = b * np.exp(2j * np.pi * 8 / 1024 * n)
    E = A + s * np.conj(synth.kk_phase(fc_step, n))
    I = np.abs(E) ** 2
    out = kk.kk_field(I, pad=float(np.mean(I)), fc_step=fc_step)
    sl = slice(1024, N - 1024)
    assert np.max(np.abs(out[sl] - s[sl])) < 1e-10 * A
    # the opposite downconversion sign leaves the signal 2 fc away
    bad = out * np.conj(kk.downconvert_phase(fc_step, n)) ** 2
    assert np.max(np.abs(bad[sl] - s[sl])) > 0.5 * b


def test_kk_reconstruction_error_falls_with_cspr():
    """KK physics: a noiseless carrier-assisted 16QAM field is
    reconstructed with an error that falls as the carrier-to-signal power
    ratio grows (fewer minimum-phase violations, smaller out-of-band
    content of ln|E|): below -30 dB at 14 dB CSPR."""
    nmse = []
    for cspr in (8.0, 14.0, 20.0):
        k = synth.make_kk_stream("dp_16qam", 8192, seed=5, cspr_db=cspr, esn0_db=30.0, noise=False)
        out = kk.kk_field(k.intensity, pad=k.dc, fc_step=k.fc_step)
        sl = slice(2048, -2048)
        e = out[sl] - k.field[sl]
        nmse.append(10 * np.log10(np.mean(np.abs(e) ** 2) / np.mean(np.abs(k.field[sl]) ** 2)))
    assert nmse[0] > nmse[1] > nmse[2]
    assert nmse[1] < -30.0


def test_codes_with_dc_added_back_give_the_intensity():
    """Sec. 2's first kernel: code * scale + DC offset is the detected
    intensity to within half a quantisation step."""
    k = synth.make_kk_stream("dp_16qam", 4096, seed=7, cspr_db=12.0, esn0_db=20.0)
    I = kk.intensity_from_codes(k.codes, k.scale, k.dc)
    assert np.max(np.abs(I - k.intensity)) <= 0.5 * k.scale * (1 + 1e-9)
