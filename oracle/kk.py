"""FP64 oracle of the Kramers-Kronig front-end (test infrastructure only).

Sec. 2 of the paper: the first kernel converts the ADC's fixed-point
samples to floating point, adds back the DC term that the AC-coupled
detector lost, and takes the square root (the field amplitude) and the
logarithm; a pair of overlap-save 1024-point FFTs then recovers the
field's phase by a frequency-domain Hilbert transform; amplitude and phase
together give the optical field, which is downconverted.  The underlying
relation (Kramers-Kronig, the paper's ref. on KK coherent detection): for a
minimum-phase field E = A + s', ln E is analytic on one side of the
spectrum, so its imaginary part (the phase) is the Hilbert transform of its
real part ln|E| = ln(I)/2.

Readings where the paper is silent (each also used by the CUDA path):

* sideband: the signal sits below the carrier (E = A + s e^{-j 2 pi fc n}),
  so ln E has only negative-frequency content and the phase is
  phi = IFFT(G * FFT(ln|E|)), G = +j on the positive bins, -j on the
  negative bins, 0 at DC and at N/2;
* overlap-save: frames of n_fft samples starting at f*(n_fft - n_ov) -
  n_ov/2, centre n_fft - n_ov samples kept (the paper's "100% overlap" read
  as n_ov = n_fft/2);
* outside the stream the AC-coupled samples are zero, i.e. the intensity
  equals the DC term;
* intensities below ``floor`` are clamped to it before the root and the
  logarithm (minimum-phase violations and noise can make them <= 0);
* carrier removal: the carrier amplitude of a frame is exp of the mean of
  ln|E| over the frame (the DC bin of its spectrum: ln A is the DC of ln E
  for a minimum-phase field whose signal leaves a gap at the carrier), and
  is subtracted from the reconstructed field before the downconversion;
* downconversion by e^{+j 2 pi fc n}, fc held as a 32-bit phase increment
  per sample (``fc_step`` = fc * 2^32), n counted from the stream start.

numpy's FFT is the only library primitive used as a step.
"""
from __future__ import annotations

import numpy as np


def intensity_from_codes(codes: np.ndarray, scale: float, dc: float) -> np.ndarray:
    """ADC codes -> photocurrent with the DC term added back (Sec. 2, first kernel)."""
    return scale * np.asarray(codes, dtype=np.float64) + dc


def hilbert_gain(n_fft: int) -> np.ndarray:
    """G[k]: +j for 0 < k < N/2, -j for N/2 < k < N, 0 at k = 0 and N/2."""
    g = np.zeros(n_fft, dtype=np.complex128)
    g[1:n_fft // 2] = 1j
    g[n_fft // 2 + 1:] = -1j
    return g


def frame_phase(l: np.ndarray) -> tuple[np.ndarray, float]:
    """One frame of ln|E| -> (phase phi over the frame, mean of ln|E|)."""
    n = l.shape[0]
    L = np.fft.fft(l)
    phi = np.fft.ifft(L * hilbert_gain(n)).real
    return phi, float(L[0].real / n)


def downconvert_phase(fc_step: int, n: np.ndarray) -> np.ndarray:
    """exp(+j 2 pi (fc_step * n mod 2^32) / 2^32)."""
    u = (np.asarray(n, dtype=np.uint64) * np.uint64(fc_step)) & np.uint64(0xFFFFFFFF)
    return np.exp(2j * np.pi * (u.astype(np.float64) / 2.0 ** 32))


def kk_field(I: np.ndarray, *, pad: float, fc_step: int, n_fft: int = 1024, n_ov: int = 512,
             floor: float = 1e-9) -> np.ndarray:
    """Intensity samples I [n] (DC included) -> downconverted signal field [n].

    ``pad`` is the intensity taken outside the stream (the DC term)."""
    I = np.asarray(I, dtype=np.float64)
    ns = I.shape[0]
    step, half = n_fft - n_ov, n_ov // 2
    Ic = np.maximum(I, floor)
    a = np.sqrt(Ic)
    l_pad = 0.5 * np.log(max(pad, floor))
    l_all = 0.5 * np.log(Ic)
    out = np.empty(ns, dtype=np.complex128)
    n_frames = (ns + step - 1) // step
    for f in range(n_frames):
        start = f * step - half
        idx = np.arange(start, start + n_fft)
        inside = (idx >= 0) & (idx < ns)
        l = np.full(n_fft, l_pad)
        l[inside] = l_all[idx[inside]]
        phi, lbar = frame_phase(l)
        A = np.exp(lbar)
        pos = np.arange(half, half + step)
        n = start + pos
        keep = n < ns
        pos, n = pos[keep], n[keep]
        E = a[n] * np.exp(1j * phi[pos]) - A
        out[n] = E * downconvert_phase(fc_step, n)
    return out


def kk_field_from_codes(codes: np.ndarray, *, scale: float, dc: float, fc_step: int,
                        n_fft: int = 1024, n_ov: int = 512, floor: float = 1e-9) -> np.ndarray:
    """The front-end from ADC codes: intensity = scale * code + dc; zero
    codes (intensity dc) outside the stream."""
    return kk_field(intensity_from_codes(codes, scale, dc), pad=dc, fc_step=fc_step,
                    n_fft=n_fft, n_ov=n_ov, floor=floor)
