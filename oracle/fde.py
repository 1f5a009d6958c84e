"""FP64 oracle of the trained static frequency-domain equaliser (test
infrastructure only).

Sec. 2 of the paper: after the Kramers-Kronig front-end, a second pair of
FFTs applies a static equaliser of 203 taps and resamples from 4 to 2
samples per symbol; the equaliser is optimised offline from a training
sequence each time acquisition starts.

Readings where the paper is silent (each also used by the CUDA path):

* the 203 taps h[t] act at the input rate, centred (delay D = (T-1)/2):
  z[n] = sum_t h[t] x[n + D - t];
* training = regularised least squares on the symbol instants: minimise
  sum_i |z[sps*i] - d_i|^2 + lam |h|^2 over the first K known symbols d,
  lam = delta * trace(R) / T with R = U^H U, U[i, t] = x[sps*i + D - t]
  (zero outside the stream), i.e. (R + lam I) h = U^H d;
* application: overlap-save frames of n_fft = 1024 input samples starting at
  f*(n_fft - n_ov) - n_ov/2; spectrum times the equaliser's response
  H[k] = sum_t h[t] e^{-j 2 pi k (t - D) / n_fft}, restricted to the output
  band k in [0, n_fft/4) U [3 n_fft/4, n_fft) (|f| < fs/4); inverse FFT;
  the centre n_fft - n_ov samples kept and every second one output
  (output m is input-rate sample 2m).

numpy's FFT and linear solve are the library primitives used as steps.
"""
from __future__ import annotations

import numpy as np


def regressors(x: np.ndarray, K: int, T: int, sps: int = 4) -> np.ndarray:
    """U [K, T], U[i, t] = x[sps*i + D - t] (0 outside the stream)."""
    x = np.asarray(x, dtype=np.complex128)
    D = (T - 1) // 2
    idx = sps * np.arange(K)[:, None] + D - np.arange(T)[None, :]
    ok = (idx >= 0) & (idx < x.shape[0])
    U = np.zeros((K, T), dtype=np.complex128)
    U[ok] = x[idx[ok]]
    return U


def train(x: np.ndarray, d: np.ndarray, T: int = 203, sps: int = 4, delta: float = 1e-6) -> np.ndarray:
    """Least-squares taps h [T] from the stream x (input rate) and the
    known symbols d [K] (symbol i at input sample sps*i)."""
    d = np.asarray(d, dtype=np.complex128)
    U = regressors(x, d.shape[0], T, sps)
    R = U.conj().T @ U
    p = U.conj().T @ d
    lam = delta * np.trace(R).real / T
    return np.linalg.solve(R + lam * np.eye(T), p)


def band(n_fft: int = 1024) -> np.ndarray:
    """1 on the output band k in [0, N/4) U [3N/4, N), 0 elsewhere."""
    b = np.zeros(n_fft)
    b[:n_fft // 4] = 1.0
    b[3 * n_fft // 4:] = 1.0
    return b


def response(h: np.ndarray, n_fft: int = 1024) -> np.ndarray:
    """H[k] = sum_t h[t] e^{-j 2 pi k (t - D) / N} on the output band, 0 off it."""
    h = np.asarray(h, dtype=np.complex128)
    T = h.shape[0]
    D = (T - 1) // 2
    k = np.arange(n_fft)[:, None]
    t = np.arange(T)[None, :]
    H = np.exp(-2j * np.pi * k * (t - D) / n_fft) @ h
    return H * band(n_fft)


def apply(x: np.ndarray, h: np.ndarray, n_fft: int = 1024, n_ov: int = 256) -> np.ndarray:
    """Input-rate stream x [n] (n even) -> equalised output [n/2] at half the rate."""
    x = np.asarray(x, dtype=np.complex128)
    ns = x.shape[0]
    step, half = n_fft - n_ov, n_ov // 2
    H = response(h, n_fft)
    out = np.empty(ns // 2, dtype=np.complex128)
    for f in range((ns + step - 1) // step):
        start = f * step - half
        idx = np.arange(start, start + n_fft)
        inside = (idx >= 0) & (idx < ns)
        fr = np.zeros(n_fft, dtype=np.complex128)
        fr[inside] = x[idx[inside]]
        z = np.fft.ifft(np.fft.fft(fr) * H)
        for pos in range(half, half + step):
            o = start + pos
            if o < ns and o % 2 == 0:
                out[o // 2] = z[pos]
    return out
