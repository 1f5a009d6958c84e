"""Offline geometric-shaping (GS) designer for the 4D 64-ary format.

Sec. 5 of the paper designs its GS constellations for the AWGN channel by a
greedy search: start from the conventional layout; alternately (a) add
Gaussian noise to one randomly chosen point and (b) swap the binary labels
of two randomly chosen points; evaluate the AWGN GMI after each move and keep
the move only if the GMI increased.  It also imposes symmetries to help the
search converge.

The paper prints no 4D 64-point table, so this module builds one with that
procedure (design Es/N0 14 dB per polarisation, the paper's GS-8 design
point for 3 bits per 2D):

* conventional start: the product of two circular (4,4) 8-QAMs (inner QPSK
  ring at 45 degrees, outer ring on the axes, radius ratio (sqrt2+sqrt6)/2,
  the equal-distance layout), one per polarisation;
* symmetry: invariance under a joint 90-degree rotation of both
  polarisations, so the 64 points are 16 orbit representatives times the
  four rotations; a label is 2 Gray-coded rotation bits (MSB side) followed
  by the 4-bit orbit label.  Moves act on orbits, so the symmetry is exact
  (a 90-degree rotation of a float is exact);
* energy: each polarisation is rescaled to unit mean energy after a move;
* GMI: Monte-Carlo with a fixed, seeded set of noise samples, so a move's
  acceptance is deterministic.

Run ``python -m paper_2108_07004_gb300.gs_design`` to rewrite
``data/gs4d64_v1.json``.  The written table is the artefact; both the CUDA
library (as an uploaded table, Sec. 2) and the tests read it.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

GRAY2 = (0, 1, 3, 2)          # rotation index k -> 2-bit Gray label
OUT = os.path.join(os.path.dirname(__file__), "data", "gs4d64_v1.json")


def star8() -> tuple[np.ndarray, np.ndarray]:
    """Inner ring (4 points at 45 + k*90 deg) and outer ring (k*90 deg)."""
    a = 1.0
    b = a * (np.sqrt(2) + np.sqrt(6)) / 2
    inner = a * np.exp(1j * (np.pi / 4 + np.pi / 2 * np.arange(4)))
    outer = b * np.exp(1j * (np.pi / 2 * np.arange(4)))
    return inner, outer


def initial_orbits() -> np.ndarray:
    """16 orbit representatives [16, 2] of the product of two star 8-QAMs.

    Every orbit of the joint 90-degree rotation has one member whose X
    component is the inner point at 45 degrees or the outer point at 0
    degrees; Y runs over all 8 points."""
    inner, outer = star8()
    ypts = np.concatenate([inner, outer])
    reps = []
    for xp in (inner[0], outer[0]):
        for yp in ypts:
            reps.append((xp, yp))
    return np.asarray(reps, dtype=np.complex128)


def expand(reps: np.ndarray, orbit_label: np.ndarray) -> np.ndarray:
    """Points [64, 2] indexed by label (rot_gray << 4 | orbit_label)."""
    pts = np.empty((64, 2), dtype=np.complex128)
    for o in range(16):
        for k in range(4):
            pts[(GRAY2[k] << 4) | int(orbit_label[o])] = reps[o] * (1j ** k)
    return pts


def normalise(reps: np.ndarray) -> np.ndarray:
    """Unit mean energy per polarisation (over the orbit representatives,
    which equals the mean over all 64 points since rotation keeps |.|)."""
    e = np.mean(np.abs(reps) ** 2, axis=0)
    return reps / np.sqrt(e)[None, :]


def gmi_awgn(pts: np.ndarray, n0: float, noise: np.ndarray) -> float:
    """Monte-Carlo AWGN GMI in bits per 4D symbol, exact LLRs.

    ``noise`` [K, 2] complex with variance n0 per polarisation."""
    m = 6
    labels = np.arange(64)
    bits = (labels[:, None] >> np.arange(m - 1, -1, -1)[None, :]) & 1     # [64, 6]
    y = pts[:, None, :] + noise[None, :, :]                                 # [64, K, 2]
    d = np.sum(np.abs(y[:, :, None, :] - pts[None, None, :, :]) ** 2, axis=-1)  # [64,K,64]
    logit = -d / n0
    total = 0.0
    for i in range(m):
        l0 = _lse(logit[:, :, bits[:, i] == 0])
        l1 = _lse(logit[:, :, bits[:, i] == 1])
        llr = l0 - l1
        sgn = 1.0 - 2.0 * bits[:, i][:, None]
        total += np.mean(np.logaddexp(0.0, -sgn * llr)) / np.log(2)
    return m - total


def _lse(x: np.ndarray) -> np.ndarray:
    mx = np.max(x, axis=-1, keepdims=True)
    return (mx + np.log(np.sum(np.exp(x - mx), axis=-1, keepdims=True)))[..., 0]


def design(esn0_db: float = 14.0, iters: int = 2000, n_noise: int = 256,
           sigma_p: float = 0.05, seed: int = 2108070043, verbose: bool = False):
    rng = np.random.Generator(np.random.PCG64(seed))
    n0 = 10 ** (-esn0_db / 10)
    w = rng.standard_normal((2, n_noise, 2))
    noise = np.sqrt(n0 / 2) * (w[0] + 1j * w[1])

    reps = normalise(initial_orbits())
    olab = np.arange(16)
    best = gmi_awgn(expand(reps, olab), n0, noise)
    gmi0 = best
    accepted = 0
    for it in range(iters):
        if it % 2 == 0:          # perturb one orbit representative
            o = int(rng.integers(16))
            step = sigma_p * (rng.standard_normal(2) + 1j * rng.standard_normal(2)) / np.sqrt(2)
            cand_reps = reps.copy()
            cand_reps[o] = cand_reps[o] + step
            cand_reps = normalise(cand_reps)
            cand_lab = olab
        else:                    # swap the labels of two orbits
            a, b = rng.choice(16, size=2, replace=False)
            cand_lab = olab.copy()
            cand_lab[a], cand_lab[b] = cand_lab[b], cand_lab[a]
            cand_reps = reps
        g = gmi_awgn(expand(cand_reps, cand_lab), n0, noise)
        if g > best:
            best, reps, olab = g, cand_reps, cand_lab
            accepted += 1
        if verbose and it % 200 == 0:
            print(f"iter {it} gmi {best:.5f} accepted {accepted}")
    return expand(reps, olab), dict(gmi_init=gmi0, gmi_final=best, accepted=accepted,
                                    iters=iters, n_noise=n_noise, sigma_p=sigma_p,
                                    seed=seed, esn0_db=esn0_db)


def table_json(pts: np.ndarray, info: dict) -> dict:
    rows = [[float(p[0].real), float(p[0].imag), float(p[1].real), float(p[1].imag)]
            for p in pts]
    # store the float32 values the GPU consumes, so both sides read identical points
    rows32 = [[float(np.float32(v)) for v in r] for r in rows]
    blob = json.dumps(rows32).encode()
    return dict(name="gs4d64", dims=4, m_bits=6, sym_order=4,
                description="4D 64-ary GS format designed by the paper's Sec. 5 "
                            "greedy AWGN-GMI search (see gs_design.py)",
                design=info, labels=list(range(64)), points=rows32,
                sha256=hashlib.sha256(blob).hexdigest())


def main():
    pts, info = design(verbose=True)
    d = table_json(pts, info)
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as f:
        json.dump(d, f, indent=1)
    print(f"wrote {OUT}: gmi {info['gmi_init']:.5f} -> {info['gmi_final']:.5f}")


if __name__ == "__main__":
    main()
