"""Seeded synthetic channel generator (untimed input side).

Produces dual-polarisation received samples shaped like a 28 GBd coherent
link: i.i.d. uniform bits mapped onto a constellation (PCG64 random numbers,
as the transmitter in Sec. 3 of the paper uses), root-raised-cosine pulse
shaping at ``sps`` samples per symbol, chromatic dispersion
H_CD(f) = exp(j*D*L*lambda^2*omega^2/(4*pi*c)), a fixed Haar-random 2x2
unitary polarisation rotation, one Wiener laser phase process common to
both polarisations, and complex AWGN.

This module is shared by the tests, the benchmark and the oracle.  It holds
none of the receiver's arithmetic: it only makes inputs.  All arithmetic is
float64; the output samples are cast to complex64.

Conventions
-----------
* Es/N0 is per polarisation per symbol; the constellation has unit mean
  energy per polarisation, so N0 = 10**(-EsN0_dB/10).
* The transmit filter G(f) = sqrt(sps * r(f)), r the raised-cosine shape,
  so that sum(g**2) == 1 and the matched-filtered, symbol-spaced samples
  reproduce the symbols exactly (Nyquist).  AWGN of complex variance N0 per
  sample therefore gives Es/N0 at the matched-filter output.
* Spectra use numpy's forward DFT sign (exp(-j 2 pi k n / N)), under which
  H_CD above delays low frequencies more than high ones for D > 0, as
  standard single-mode fibre at 1550 nm does.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft

C_LIGHT = 299_792_458.0
LAMBDA_1550 = 1550e-9
SEED_BASE = 2108070040

_DATA = os.path.join(os.path.dirname(__file__), "data")


def stream_seed(cfg: int, point: int = 0) -> int:
    """Seed convention for workload ``cfg`` and sweep point ``point``."""
    return SEED_BASE + 10 * cfg + point


# ---------------------------------------------------------------------------
# transmitter constellations (Tx mapping only)
# ---------------------------------------------------------------------------

@dataclass
class TxFormat:
    name: str
    dims: int            # 2: the same 2D table on each polarisation; 4: joint 4D
    points: np.ndarray   # dims==2: [M] complex; dims==4: [M, 2] complex; index == label
    bits_per_4d: int     # bits per 4D symbol (both polarisations)


def _gray_pam_levels(nbits: int) -> np.ndarray:
    """Amplitude for each PAM label, Gray coded, label MSB = sign (0 -> +)."""
    n = 1 << nbits
    levels = np.empty(n)
    # position p (0 = most positive) carries Gray code p ^ (p >> 1)
    for p in range(n):
        g = p ^ (p >> 1)
        levels[g] = (n - 1) - 2 * p
    return levels


def tx_qam_gray(m_pol: int) -> TxFormat:
    """Square Gray QAM with ``m_pol`` bits per polarisation (2: QPSK, 4: 16QAM)."""
    h = m_pol // 2
    lv = _gray_pam_levels(h)
    pts = np.empty(1 << m_pol, dtype=np.complex128)
    for lab in range(1 << m_pol):
        pts[lab] = lv[lab >> h] + 1j * lv[lab & ((1 << h) - 1)]
    pts /= np.sqrt(np.mean(np.abs(pts) ** 2))
    name = {2: "dp_qpsk", 4: "dp_16qam"}.get(m_pol, f"dp_{1 << m_pol}qam")
    return TxFormat(name, 2, pts, 2 * m_pol)


def tx_table4d(path: str) -> TxFormat:
    """Joint 4D table from a JSON file holding ``points`` as [M][4] reals
    (x_re, x_im, y_re, y_im) and ``labels`` (a permutation of 0..M-1)."""
    with open(path) as f:
        d = json.load(f)
    p = np.asarray(d["points"], dtype=np.float64)
    lab = np.asarray(d["labels"], dtype=np.int64)
    pts = np.empty((len(lab), 2), dtype=np.complex128)
    pts[lab, 0] = p[:, 0] + 1j * p[:, 1]
    pts[lab, 1] = p[:, 2] + 1j * p[:, 3]
    return TxFormat(d.get("name", "table4d"), 4, pts, int(np.log2(len(lab))))


def tx_table2d(path: str) -> TxFormat:
    """2D table (the same on each polarisation) from a JSON file holding
    ``points`` as [M][2] reals and ``labels`` (a permutation of 0..M-1)."""
    with open(path) as f:
        d = json.load(f)
    p = np.asarray(d["points"], dtype=np.float64)
    lab = np.asarray(d["labels"], dtype=np.int64)
    pts = np.empty(len(lab), dtype=np.complex128)
    pts[lab] = p[:, 0] + 1j * p[:, 1]
    return TxFormat(d.get("name", "table2d"), 2, pts, 2 * int(np.log2(len(lab))))


def tx_format(name: str) -> TxFormat:
    if name == "dp_qpsk":
        return tx_qam_gray(2)
    if name == "dp_16qam":
        return tx_qam_gray(4)
    if name == "dp_64qam":
        return tx_qam_gray(6)
    if name in ("gs8", "gs128"):
        return tx_table2d(os.path.join(_DATA, f"{name}_v1.json"))
    if name == "gs4d64":
        return tx_table4d(os.path.join(_DATA, "gs4d64_v1.json"))
    raise ValueError(f"unknown format {name!r}")


def bits_to_symbols(fmt: TxFormat, bits: np.ndarray) -> np.ndarray:
    """bits [N, m] (MSB first; for 2D formats X bits then Y bits) -> [2, N]."""
    n, m = bits.shape
    w = (1 << np.arange(m - 1, -1, -1)).astype(np.int64)
    if fmt.dims == 4:
        lab = bits.astype(np.int64) @ w
        return fmt.points[lab].T.copy()
    h = m // 2
    wx = (1 << np.arange(h - 1, -1, -1)).astype(np.int64)
    lx = bits[:, :h].astype(np.int64) @ wx
    ly = bits[:, h:].astype(np.int64) @ wx
    return np.stack([fmt.points[lx], fmt.points[ly]])


# ---------------------------------------------------------------------------
# channel
# ---------------------------------------------------------------------------

def raised_cosine_shape(f: np.ndarray, symbol_rate: float, rolloff: float) -> np.ndarray:
    """Normalised raised-cosine spectrum r(f) in [0, 1]."""
    af = np.abs(f)
    f1 = (1 - rolloff) * symbol_rate / 2
    f2 = (1 + rolloff) * symbol_rate / 2
    r = np.zeros_like(af)
    r[af <= f1] = 1.0
    band = (af > f1) & (af <= f2)
    if rolloff > 0:
        r[band] = 0.5 * (1 + np.cos(np.pi / (rolloff * symbol_rate) * (af[band] - f1)))
    return r


def cd_channel_response(f: np.ndarray, cd_ps_per_nm: float,
                        wavelength: float = LAMBDA_1550) -> np.ndarray:
    """Fibre response exp(j*D*L*lambda^2*omega^2/(4*pi*c)), D*L in ps/nm."""
    dl = cd_ps_per_nm * 1e-3                     # ps/nm -> s/m
    w = 2 * np.pi * f
    return np.exp(1j * dl * wavelength ** 2 * w ** 2 / (4 * np.pi * C_LIGHT))


def haar_unitary(rng: np.random.Generator) -> np.ndarray:
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


@dataclass
class Stream:
    rx: np.ndarray        # [2, sps*N] complex64, pol-major
    bits: np.ndarray      # [N, m] uint8
    sym: np.ndarray       # [2, N] complex128 transmitted symbols
    J: np.ndarray         # [2, 2] polarisation rotation
    phase: np.ndarray     # [sps*N] float64 laser phase per sample
    n0: float
    fmt: TxFormat


def make_stream(fmt: TxFormat | str, n_sym: int, *, seed: int, esn0_db: float,
                cd_ps_per_nm: float, linewidth_ts: float, sps: int = 2,
                rolloff: float = 0.1, symbol_rate: float = 28e9,
                wavelength: float = LAMBDA_1550, rotation: bool = True,
                noise: bool = True, pad_samples: int = 4096,
                phase0: float | None = None,
                iq_imbalance: tuple[float, float] | None = None) -> Stream:
    """Generate one seeded stream of ``n_sym`` 4D symbols.

    ``iq_imbalance`` = (gain error eps, phase error phi in rad) of the
    transmitter's IQ modulators: each polarisation's symbols become
    alpha s + beta conj(s), alpha = (1 + (1 + eps) e^{-j phi}) / 2,
    beta = (1 - (1 + eps) e^{j phi}) / 2 (before the real pulse shaping).
    The reference symbols and bits stay the ideal ones."""
    if isinstance(fmt, str):
        fmt = tx_format(fmt)
    rng = np.random.Generator(np.random.PCG64(seed))
    m = fmt.bits_per_4d
    bits = rng.integers(0, 2, size=(n_sym, m), dtype=np.uint8)
    sym = bits_to_symbols(fmt, bits)
    J = haar_unitary(rng) if rotation else np.eye(2, dtype=np.complex128)

    ns = sps * n_sym
    nfft = sfft.next_fast_len(ns + pad_samples)
    u = np.zeros((2, nfft), dtype=np.complex128)
    if iq_imbalance is not None:
        eps, phi = iq_imbalance
        alpha = (1 + (1 + eps) * np.exp(-1j * phi)) / 2
        beta = (1 - (1 + eps) * np.exp(1j * phi)) / 2
        u[:, 0:ns:sps] = alpha * sym + beta * np.conj(sym)
    else:
        u[:, 0:ns:sps] = sym
    f = sfft.fftfreq(nfft, d=1.0 / (sps * symbol_rate))
    g = np.sqrt(sps * raised_cosine_shape(f, symbol_rate, rolloff))
    h = g * cd_channel_response(f, cd_ps_per_nm, wavelength)
    tx = sfft.ifft(sfft.fft(u, axis=1) * h, axis=1)[:, :ns]
    sig = J @ tx

    inc = rng.standard_normal(ns) * np.sqrt(2 * np.pi * linewidth_ts / sps)
    th0 = rng.uniform(-np.pi, np.pi) if phase0 is None else phase0
    phase = th0 + np.cumsum(inc) - inc[0]
    sig = sig * np.exp(1j * phase)[None, :]

    n0 = 10.0 ** (-esn0_db / 10.0)
    if noise:
        w = rng.standard_normal((2, 2, ns))
        sig = sig + np.sqrt(n0 / 2) * (w[0] + 1j * w[1])
    return Stream(sig.astype(np.complex64), bits, sym, J, phase, n0, fmt)


def make_batch(fmt: TxFormat | str, n_sym: int, seeds, esn0_dbs, **kw):
    """Several independent streams of equal length; returns (rx [S,2,sps*N]
    complex64, list of Stream)."""
    streams = [make_stream(fmt, n_sym, seed=s, esn0_db=e, **kw)
               for s, e in zip(seeds, esn0_dbs)]
    return np.stack([s.rx for s in streams]), streams


# ---- learned demapper: seeded initial weights ------------------------------
MLP_LAYERS = ((128, 4), (128, 128), (6, 128))   # (outputs, inputs) of each layer


def mlp_init_params(seed: int) -> np.ndarray:
    """Initial parameters of the learned demapper's MLP 4 -> 128 -> 128 -> 6,
    float32 in the library's order (W1, b1, W2, b2, W3, b3): weights drawn
    uniformly in +-sqrt(6 / fan_in) (He), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for n_out, n_in in MLP_LAYERS:
        lim = np.sqrt(6.0 / n_in)
        parts.append(rng.uniform(-lim, lim, size=(n_out, n_in)).astype(np.float32).ravel())
        parts.append(np.zeros(n_out, np.float32))
    return np.concatenate(parts)


# ---- Kramers-Kronig (single-polarisation, carrier-assisted) signals --------

@dataclass
class KKStream:
    codes: np.ndarray      # [sps*N] int16 ADC codes of the AC-coupled photocurrent
    intensity: np.ndarray  # [sps*N] float64 photocurrent before AC coupling
    scale: float           # photocurrent per ADC code
    dc: float              # mean photocurrent (the term the AC coupling removed)
    fc_step: int           # carrier offset from the signal centre, cycles/sample * 2^32
    carrier: float         # carrier amplitude A
    field: np.ndarray      # [sps*N] complex128 noiseless signal s at baseband
    sym: np.ndarray        # [N] complex128 transmitted symbols
    bits: np.ndarray       # [N, m_pol] uint8
    n0: float
    sps: int


def kk_phase(fc_step: int, n: np.ndarray) -> np.ndarray:
    """exp(j 2 pi (fc_step * n mod 2^32) / 2^32): the carrier offset as a
    32-bit phase increment per sample."""
    u = (np.asarray(n, dtype=np.uint64) * np.uint64(fc_step)) & np.uint64(0xFFFFFFFF)
    return np.exp(2j * np.pi * (u.astype(np.float64) / 2.0 ** 32))


def make_kk_stream(fmt: TxFormat | str, n_sym: int, *, seed: int, cspr_db: float,
                   esn0_db: float, sps: int = 4, rolloff: float = 0.01, gap: float = 0.011,
                   adc_bits: int = 12, noise: bool = True, pad_samples: int = 4096) -> KKStream:
    """One seeded single-polarisation signal for Kramers-Kronig detection.

    The transmitter places the RRC-shaped signal s (unit-energy symbols,
    ``sps`` samples per symbol) below a real carrier A: the optical field is
    E = A + s * exp(-j 2 pi fc n) with fc = ((1 + rolloff)/2 + gap)/sps
    cycles per sample (held as a 32-bit phase increment), so that the
    carrier sits ``gap`` symbol rates above the signal's upper band edge
    (Sec. 3: 1 GBd, roll-off 0.01, carrier 11 MHz above the band).
    CSPR = A^2 / mean|s|^2.  Complex AWGN of variance N0 per sample
    (N0 = 10^(-EsN0/10), the matched-filter convention of ``make_stream``)
    is added to the field, a photodiode detects I = |E + n|^2, the AC
    coupling removes its mean and an ADC of ``adc_bits`` bits samples it
    with a full scale of 1.1 max|I - mean I|.  For 2D formats only (the
    symbols of the first polarisation of the 2D table)."""
    if isinstance(fmt, str):
        fmt = tx_format(fmt)
    if fmt.dims != 2:
        raise ValueError("KK signals use a 2D format")
    rng = np.random.Generator(np.random.PCG64(seed))
    m_pol = fmt.bits_per_4d // 2
    bits = rng.integers(0, 2, size=(n_sym, m_pol), dtype=np.uint8)
    w = (1 << np.arange(m_pol - 1, -1, -1)).astype(np.int64)
    sym = fmt.points[bits.astype(np.int64) @ w]

    ns = sps * n_sym
    nfft = sfft.next_fast_len(ns + pad_samples)
    u = np.zeros(nfft, dtype=np.complex128)
    u[0:ns:sps] = sym
    f = sfft.fftfreq(nfft, d=1.0 / sps)                 # in symbol rates
    g = np.sqrt(sps * raised_cosine_shape(f, 1.0, rolloff))
    s = sfft.ifft(sfft.fft(u) * g)[:ns]

    fc = ((1 + rolloff) / 2 + gap) / sps
    fc_step = int(round(fc * 2.0 ** 32))
    p_s = 1.0 / sps                                     # mean |s|^2 per sample
    A = float(np.sqrt(10.0 ** (cspr_db / 10.0) * p_s))
    n_idx = np.arange(ns)
    E = A + s * np.conj(kk_phase(fc_step, n_idx))
    n0 = 10.0 ** (-esn0_db / 10.0)
    if noise:
        wn = rng.standard_normal((2, ns))
        E = E + np.sqrt(n0 / 2) * (wn[0] + 1j * wn[1])
    I = np.abs(E) ** 2
    dc = float(np.mean(I))
    ac = I - dc
    full = (1 << (adc_bits - 1)) - 1
    scale = float(1.1 * np.max(np.abs(ac)) / full)
    codes = np.clip(np.round(ac / scale), -full - 1, full).astype(np.int16)
    return KKStream(codes, I, scale, dc, fc_step, A, s, sym, bits, n0, sps)
