"""Offline geometric-shaping (GS) designer for the 2D GS-8 and GS-128 formats.

Sec. 5 of the paper designs GS-8 (for 14 dB SNR) and GS-128 (for 20 dB) for
the AWGN channel by a greedy search: from the conventional layout,
alternately (a) add Gaussian noise to one randomly chosen point and (b) swap
the binary labels of two randomly chosen points; a move is kept only if the
AWGN GMI increases; symmetries are imposed to help convergence.  The paper
prints neither table, so this module builds both with that procedure:

* conventional starts: the circular (4,4) 8-QAM (inner QPSK ring at 45
  degrees, outer ring on the axes, radius ratio (sqrt2 + sqrt6)/2) and the
  cross 128-QAM (odd coordinates up to +-11 without the 16 corner points);
* symmetry: invariance under a 90-degree rotation, so the M points are M/4
  orbit representatives times the four rotations; a label is 2 Gray-coded
  rotation bits (MSB side) followed by the orbit label.  Moves act on
  orbits, so the symmetry is exact and the phase search can use S = 4;
* energy: unit mean energy after every move;
* GMI: Monte-Carlo with a fixed, seeded set of noise samples per point, so a
  move's acceptance is deterministic.

Run ``python -m paper_2108_07004_gb300.gs2d_design`` to rewrite
``data/gs8_v1.json`` and ``data/gs128_v1.json``.  The written tables are the
artefacts the tests and the library read.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

GRAY2 = (0, 1, 3, 2)          # rotation index k -> 2-bit Gray label
DATA = os.path.join(os.path.dirname(__file__), "data")


def star8_orbits() -> np.ndarray:
    """Orbit representatives of the circular (4,4) 8-QAM: inner at 45 deg, outer at 0 deg."""
    a = 1.0
    b = a * (np.sqrt(2) + np.sqrt(6)) / 2
    return np.array([a * np.exp(1j * np.pi / 4), b + 0j])


def cross128_orbits() -> np.ndarray:
    """The 32 first-quadrant points of the cross 128-QAM (odd coordinates
    1..11, without those with both coordinates above 8), in the order of
    their conventional quasi-Gray orbit labels (``cross128_labels``)."""
    lv = np.arange(1, 12, 2)
    reps = [x + 1j * y for x in lv for y in lv if not (x > 8 and y > 8)]
    lab = [cross128_label(int(r.real), int(r.imag)) for r in reps]
    out = np.empty(32, dtype=np.complex128)
    out[lab] = reps
    return out


def cross128_label(x: int, y: int) -> int:
    """Quasi-Gray 5-bit orbit label of the first-quadrant cross point (x, y):
    the inner 4 x 4 block carries 2-bit Gray codes of both coordinates;
    the strips beyond 8 set the fifth bit and mirror the block's codes
    across the line 8 (right strip: x; upper strip: y, with its two Gray
    bits and the x code exchanged so that all 32 labels differ)."""
    g = (0, 1, 3, 2)
    ix, iy = (x - 1) // 2, (y - 1) // 2
    if x < 8 and y < 8:
        return (g[ix] << 2) | g[iy]
    if x > 8:                                   # ix in {4, 5} mirrored to {3, 2}
        return 16 | (g[7 - ix] << 2) | g[iy]
    return 16 | (g[7 - iy] - 2) << 2 | g[ix]   # g[3] - 2 = 0, g[2] - 2 = 1


def expand(reps: np.ndarray, olab: np.ndarray) -> np.ndarray:
    """Points [M] indexed by label (rot_gray << b | orbit_label), M = 4 * len(reps)."""
    n = reps.shape[0]
    b = int(np.log2(n))
    pts = np.empty(4 * n, dtype=np.complex128)
    for o in range(n):
        for k in range(4):
            pts[(GRAY2[k] << b) | int(olab[o])] = reps[o] * (1j ** k)
    return pts


def normalise(reps: np.ndarray) -> np.ndarray:
    return reps / np.sqrt(np.mean(np.abs(reps) ** 2))


def gmi_awgn(pts: np.ndarray, n0: float, noise: np.ndarray) -> float:
    """Monte-Carlo AWGN GMI in bits per 2D symbol with exact LLRs; noise
    [K] complex of variance n0, added to every point.  Per received sample
    the exponentials relative to the nearest point are summed over the
    label subsets of each bit by one product with the bit masks."""
    M = pts.shape[0]
    m = int(np.log2(M))
    bits = ((np.arange(M)[:, None] >> np.arange(m - 1, -1, -1)[None, :]) & 1).astype(np.float64)
    y = (pts[:, None] + noise[None, :]).reshape(-1)                    # [M K]
    d = np.abs(y[:, None] - pts[None, :]) ** 2 / n0                   # [M K, M]
    e = np.exp(-(d - d.min(axis=1, keepdims=True)))
    s1 = np.maximum(e @ bits, 1e-300)
    s0 = np.maximum(e @ (1.0 - bits), 1e-300)
    llr = np.log(s0) - np.log(s1)                                      # [M K, m]
    tx = np.repeat(bits, noise.shape[0], axis=0)                       # the sent point's bits
    return m - float(np.mean(np.sum(np.logaddexp(0.0, -(1.0 - 2.0 * tx) * llr), axis=1))) / np.log(2)


def noise_set(esn0_db: float, n_noise: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((2, n_noise))
    return np.sqrt(10 ** (-esn0_db / 10) / 2) * (w[0] + 1j * w[1])


def design(reps0: np.ndarray, esn0_db: float, iters: int, n_noise: int, sigma_p: float, seed: int,
           verbose: bool = False):
    rng = np.random.Generator(np.random.PCG64(seed))
    n0 = 10 ** (-esn0_db / 10)
    noise = noise_set(esn0_db, n_noise, seed + 1)
    n = reps0.shape[0]
    reps = normalise(reps0.copy())
    olab = np.arange(n)
    best = gmi_awgn(expand(reps, olab), n0, noise)
    gmi0, accepted = best, 0
    for it in range(iters):
        if it % 2 == 0 or n < 2:       # perturb one orbit representative
            o = int(rng.integers(n))
            cand = reps.copy()
            cand[o] += sigma_p * (rng.standard_normal() + 1j * rng.standard_normal()) / np.sqrt(2)
            cand, clab = normalise(cand), olab
        else:                          # swap the labels of two orbits
            a, b = rng.choice(n, size=2, replace=False)
            clab = olab.copy()
            clab[a], clab[b] = clab[b], clab[a]
            cand = reps
        g = gmi_awgn(expand(cand, clab), n0, noise)
        if g > best:
            best, reps, olab = g, cand, clab
            accepted += 1
        if verbose and it % 250 == 0:
            print(f"iter {it} gmi {best:.5f} accepted {accepted}")
    return expand(reps, olab), dict(gmi_init=gmi0, gmi_final=best, accepted=accepted, iters=iters,
                                    n_noise=n_noise, sigma_p=sigma_p, seed=seed, esn0_db=esn0_db)


def table_json(name: str, pts: np.ndarray, info: dict, start: str) -> dict:
    rows32 = [[float(np.float32(p.real)), float(np.float32(p.imag))] for p in pts]
    blob = json.dumps(rows32).encode()
    M = pts.shape[0]
    return dict(name=name, dims=2, m_bits=int(np.log2(M)), sym_order=4,
                description=f"2D {M}-ary GS format designed by the paper's Sec. 5 greedy AWGN-GMI "
                            f"search from the {start} (see gs2d_design.py)",
                design=info, labels=list(range(M)), points=rows32,
                sha256=hashlib.sha256(blob).hexdigest())


SPECS = {
    "gs8": dict(start="circular (4,4) 8-QAM", reps=star8_orbits, esn0_db=14.0, iters=600, n_noise=4096,
                sigma_p=0.05, seed=2108070044),
    "gs128": dict(start="cross 128-QAM", reps=cross128_orbits, esn0_db=20.0, iters=4000, n_noise=96,
                  sigma_p=0.03, seed=2108070045),
}


def main():
    for name, sp in SPECS.items():
        pts, info = design(sp["reps"](), sp["esn0_db"], sp["iters"], sp["n_noise"], sp["sigma_p"], sp["seed"],
                           verbose=True)
        out = os.path.join(DATA, f"{name}_v1.json")
        with open(out, "w") as f:
            json.dump(table_json(name, pts, info, sp["start"]), f, indent=1)
        print(f"wrote {out}: gmi {info['gmi_init']:.5f} -> {info['gmi_final']:.5f}")


if __name__ == "__main__":
    main()
