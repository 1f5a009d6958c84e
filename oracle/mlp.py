"""Learned demapper in FP64: an MLP 4 -> 128 -> 128 -> 6 with GELU, trained
with binary cross-entropy on the bits and Adam.  TEST INFRASTRUCTURE ONLY
(see the package docstring).

The network is the learned alternative to the exact log-sum-exp demapper
(paper Sec. 5 designs the constellation with the GMI of exact bitwise
demapping; the learned form is judged by its GMI gap to it).

Readings (the paper is silent on a learned demapper):
* Input: the de-rotated 4D symbol x = (Re z_X, Im z_X, Re z_Y, Im z_Y).
* Output: o = sigma^2 * LLR (about d_1^2 - d_0^2, which does not depend on
  the SNR), so LLR = o / sigma^2 with the block's decision-directed sigma^2;
  LLR > 0 means bit 0, bits MSB first as the exact demapper.
* Loss: mean over symbols and bits of softplus(-(1 - 2b) LLR), the binary
  cross-entropy of P(b = 0) = sigmoid(LLR).
* GELU(a) = a Phi(a) (the exact form with the normal CDF Phi).
* "BF16 weights": every layer computes with its weights rounded to bfloat16
  (round to nearest, ties to even) from float32 master weights; activations
  and accumulation stay in floating point of higher precision.
* Adam with beta1 0.9, beta2 0.999, eps 1e-8 and bias correction.

Parameter vector order (float32 on the library side): W1 [128][4], b1 [128],
W2 [128][128], b2 [128], W3 [6][128], b3 [6].

Pins (tests/test_oracle_mlp.py): GELU identities and derivative, the
backward pass against central finite differences of the loss, the BCE value
at LLR 0, Adam's first step in closed form, bfloat16 rounding of known
values, and a small training run that approaches the exact demapper's GMI.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import erf

from paper_2108_07004_gb300 import synth

H = 128
N_IN, N_OUT = 4, 6
SHAPES = [("W1", (H, N_IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
          ("W3", (N_OUT, H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    """Split a parameter vector into named arrays (views)."""
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed: int) -> np.ndarray:
    """Initial float32 parameters from the shared seeded generator (He
    uniform weights, zero biases); drawn random numbers are inputs."""
    th = synth.mlp_init_params(seed)
    assert th.size == N_PARAMS
    return th


def bf16_round(a: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def compute_weights(theta32: np.ndarray) -> dict:
    """The weights the layers use: bfloat16-rounded W, float32 biases (FP64)."""
    p = unpack(np.asarray(theta32, dtype=np.float32))
    return {k: (bf16_round(v) if k.startswith("W") else v).astype(np.float64) for k, v in p.items()}


def gelu(a):
    return 0.5 * a * (1.0 + erf(a / math.sqrt(2.0)))


def gelu_grad(a):
    return 0.5 * (1.0 + erf(a / math.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)


def softplus(t):
    return np.maximum(t, 0.0) + np.log1p(np.exp(-np.abs(t)))


def sigmoid(t):
    return 0.5 * (1.0 + np.tanh(0.5 * t))


@dataclass
class Cache:
    x: np.ndarray
    a1: np.ndarray
    h1: np.ndarray
    a2: np.ndarray
    h2: np.ndarray
    o: np.ndarray


def forward(w: dict, x: np.ndarray) -> tuple[np.ndarray, Cache]:
    """o [N, 6] = sigma^2 * LLR for inputs x [N, 4]."""
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ w["W1"].T + w["b1"]
    h1 = gelu(a1)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = gelu(a2)
    o = h2 @ w["W3"].T + w["b3"]
    return o, Cache(x, a1, h1, a2, h2, o)


def llr(w: dict, x: np.ndarray, sigma2: np.ndarray) -> np.ndarray:
    o, _ = forward(w, x)
    return o / np.asarray(sigma2, dtype=np.float64)[:, None]


def loss_and_grad(w: dict, x: np.ndarray, sigma2: np.ndarray, bits: np.ndarray):
    """Mean BCE over the N x 6 bits and its gradient (dict like w)."""
    o, c = forward(w, x)
    s2 = np.asarray(sigma2, dtype=np.float64)[:, None]
    L = o / s2
    sgn = 1.0 - 2.0 * np.asarray(bits, dtype=np.float64)      # +1 for bit 0, -1 for bit 1
    n_el = L.size
    loss = float(np.sum(softplus(-sgn * L)) / n_el)
    dL = -sgn * sigmoid(-sgn * L) / n_el                        # d loss / d LLR
    do = dL / s2
    g = {"W3": do.T @ c.h2, "b3": do.sum(axis=0)}
    dh2 = do @ w["W3"]
    da2 = dh2 * gelu_grad(c.a2)
    g["W2"] = da2.T @ c.h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ w["W2"]
    da1 = dh1 * gelu_grad(c.a1)
    g["W1"] = da1.T @ c.x
    g["b1"] = da1.sum(axis=0)
    return loss, g


@dataclass
class Adam:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    t: int = 0
    m: np.ndarray | None = None
    v: np.ndarray | None = None

    def step(self, theta: np.ndarray, grad: np.ndarray) -> np.ndarray:
        """One Adam update of the parameter vector (returns the new vector)."""
        if self.m is None:
            self.m = np.zeros_like(grad)
            self.v = np.zeros_like(grad)
        self.t += 1
        self.m = self.beta1 * self.m + (1 - self.beta1) * grad
        self.v = self.beta2 * self.v + (1 - self.beta2) * grad * grad
        mh = self.m / (1 - self.beta1 ** self.t)
        vh = self.v / (1 - self.beta2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def train(theta32: np.ndarray, x: np.ndarray, sigma2: np.ndarray, bits: np.ndarray, *,
          batch: int, steps: int, lr: float = 1e-3, seed: int = 0) -> tuple[np.ndarray, list]:
    """Adam on float32 master weights, batches drawn by a seeded permutation
    per epoch; returns the master weights and the losses."""
    rng = np.random.default_rng(seed)
    opt = Adam(lr=lr)
    theta = np.asarray(theta32, dtype=np.float32).astype(np.float64)
    n = x.shape[0]
    perm, pos, losses = rng.permutation(n), 0, []
    for _ in range(steps):
        if pos + batch > n:
            perm, pos = rng.permutation(n), 0
        idx = perm[pos:pos + batch]
        pos += batch
        w = compute_weights(theta.astype(np.float32))
        loss, g = loss_and_grad(w, x[idx], sigma2[idx], bits[idx])
        losses.append(loss)
        theta = opt.step(theta, pack(g)).astype(np.float32).astype(np.float64)
    return theta.astype(np.float32), losses
