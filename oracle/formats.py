"""Oracle-side constellation tables (test infrastructure only).

The paper's receiver makes decisions from an uploaded table of constellation
points and their bit labels and assumes no symmetry of the format (Sec. 2).
Built here independently of the CUDA library:

* DP-QPSK and DP-16QAM: Gray-mapped square QAM applied to each
  polarisation, labels MSB first, bit 0 on the positive side of each axis;
* the 4D 64-ary GS format: read from the designed table file (the paper
  prints no coordinates; see ``paper_2108_07004_gb300/gs_design.py``).
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np

_TABLE = os.path.join(os.path.dirname(__file__), os.pardir,
                      "paper_2108_07004_gb300", "data", "gs4d64_v1.json")


@dataclass
class OracleFormat:
    name: str
    dims: int              # 2: per-polarisation table; 4: joint 4D table
    points: np.ndarray     # dims 2: [M] complex128; dims 4: [M, 2]; row index == label
    m_pol: int             # bits per polarisation symbol (dims 2) or 0
    m: int                 # bits per 4D symbol
    sym_order: int = 4     # rotational symmetry used by the phase search

    @property
    def M(self) -> int:
        return self.points.shape[0]

    def bit_table(self) -> np.ndarray:
        """[M, bits per table entry] label bits, MSB first."""
        nb = self.m_pol if self.dims == 2 else self.m
        lab = np.arange(self.M)
        return ((lab[:, None] >> np.arange(nb - 1, -1, -1)[None, :]) & 1).astype(np.uint8)

    def cma_radius2(self) -> float:
        """R^2 = E|s|^4 / E|s|^2 of the per-polarisation marginal (CMA)."""
        s = self.points.reshape(-1)
        return float(np.mean(np.abs(s) ** 4) / np.mean(np.abs(s) ** 2))

    def symbols_from_bits(self, bits: np.ndarray) -> np.ndarray:
        """[N, m] bits -> [2, N] complex symbols."""
        bits = np.asarray(bits, dtype=np.int64)
        if self.dims == 4:
            lab = np.zeros(bits.shape[0], dtype=np.int64)
            for i in range(self.m):
                lab = lab * 2 + bits[:, i]
            return self.points[lab].T.copy()
        out = np.empty((2, bits.shape[0]), dtype=np.complex128)
        for p in range(2):
            lab = np.zeros(bits.shape[0], dtype=np.int64)
            for i in range(self.m_pol):
                lab = lab * 2 + bits[:, p * self.m_pol + i]
            out[p] = self.points[lab]
        return out


def _qpsk() -> OracleFormat:
    a = 1 / np.sqrt(2)
    # label b0 b1: b0 -> sign of I, b1 -> sign of Q, bit 0 = positive
    pts = np.array([a + 1j * a, a - 1j * a, -a + 1j * a, -a - 1j * a])
    return OracleFormat("dp_qpsk", 2, pts, 2, 4)


def _qam16() -> OracleFormat:
    # per-axis Gray: 00 -> +3, 01 -> +1, 11 -> -1, 10 -> -3
    lev = {0b00: 3.0, 0b01: 1.0, 0b11: -1.0, 0b10: -3.0}
    pts = np.empty(16, dtype=np.complex128)
    for lab in range(16):
        pts[lab] = lev[lab >> 2] + 1j * lev[lab & 3]
    pts /= np.sqrt(10.0)
    return OracleFormat("dp_16qam", 2, pts, 4, 8)


def _qam64() -> OracleFormat:
    # per-axis Gray over 8 levels, bit 0 of the first axis bit on the positive side:
    # 000 +7, 001 +5, 011 +3, 010 +1, 110 -1, 111 -3, 101 -5, 100 -7
    lev = {0b000: 7.0, 0b001: 5.0, 0b011: 3.0, 0b010: 1.0, 0b110: -1.0, 0b111: -3.0, 0b101: -5.0, 0b100: -7.0}
    pts = np.empty(64, dtype=np.complex128)
    for lab in range(64):
        pts[lab] = lev[lab >> 3] + 1j * lev[lab & 7]
    pts /= np.sqrt(42.0)
    return OracleFormat("dp_64qam", 2, pts, 6, 12)


def _gs2d(name: str) -> OracleFormat:
    """A 2D table file (``points`` [M][2], ``labels``), used on each polarisation."""
    with open(os.path.join(os.path.dirname(_TABLE), f"{name}_v1.json")) as f:
        d = json.load(f)
    p = np.asarray(d["points"], dtype=np.float64)
    lab = np.asarray(d["labels"], dtype=np.int64)
    pts = np.empty(len(lab), dtype=np.complex128)
    pts[lab] = p[:, 0] + 1j * p[:, 1]
    mp = int(d["m_bits"])
    return OracleFormat(name, 2, pts, mp, 2 * mp, int(d.get("sym_order", 4)))


def _gs4d64(path: str = _TABLE) -> OracleFormat:
    with open(path) as f:
        d = json.load(f)
    p = np.asarray(d["points"], dtype=np.float64)
    lab = np.asarray(d["labels"], dtype=np.int64)
    pts = np.empty((64, 2), dtype=np.complex128)
    pts[lab, 0] = p[:, 0] + 1j * p[:, 1]
    pts[lab, 1] = p[:, 2] + 1j * p[:, 3]
    return OracleFormat("gs4d64", 4, pts, 0, 6, int(d.get("sym_order", 4)))


def oracle_format(name: str) -> OracleFormat:
    if name == "dp_qpsk":
        return _qpsk()
    if name == "dp_16qam":
        return _qam16()
    if name == "gs4d64":
        return _gs4d64()
    if name == "dp_64qam":
        return _qam64()
    if name in ("gs8", "gs128"):
        return _gs2d(name)
    raise ValueError(name)
