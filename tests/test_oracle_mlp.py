"""Pins of the oracle's learned demapper (MLP 4 -> 128 -> 128 -> 6)."""
import math

import numpy as np
import pytest

from oracle import chain, mlp, oracle_format


def _awgn(n, esn0, seed):
    fmt = oracle_format("gs4d64")
    r = np.random.default_rng(seed)
    bits = r.integers(0, 2, size=(n, 6), dtype=np.uint8)
    s = fmt.symbols_from_bits(bits)
    n0 = 10 ** (-esn0 / 10)
    z = s + math.sqrt(n0 / 2) * (r.standard_normal(s.shape) + 1j * r.standard_normal(s.shape))
    x = np.stack([z[0].real, z[0].imag, z[1].real, z[1].imag], axis=1)
    return x, np.full(n, n0), bits, z


def test_gelu_identities_and_derivative():
    a = np.linspace(-6, 6, 241)
    g = mlp.gelu(a)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert np.max(np.abs(g - mlp.gelu(-a) - a)) < 1e-14            # x Phi(x) + x Phi(-x) = x
    assert abs(mlp.gelu(np.array([40.0]))[0] - 40.0) < 1e-12
    assert abs(mlp.gelu(np.array([-40.0]))[0]) < 1e-12
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    h = 1e-5
    num = (mlp.gelu(a + h) - mlp.gelu(a - h)) / (2 * h)
    assert np.max(np.abs(num - mlp.gelu_grad(a))) < 1e-9


def test_bf16_rounding_known_values():
    v = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -16, -2.5, 0.0], np.float32)
    r = mlp.bf16_round(v)
    assert list(r) == [1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -2.5, 0.0]   # ties to even
    a = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 3
    b = mlp.bf16_round(a)
    assert np.all((b.view(np.uint32) & 0xFFFF) == 0)                    # representable
    ulp = 2.0 ** (np.floor(np.log2(np.abs(a))) - 7)
    assert np.all(np.abs(b - a) <= 0.5 * ulp)


def test_bce_is_ln2_at_zero_llr():
    w = mlp.compute_weights(np.zeros(mlp.N_PARAMS, np.float32))
    x, s2, bits, _ = _awgn(64, 10.0, 1)
    loss, _ = mlp.loss_and_grad(w, x, s2, bits)
    assert abs(loss - math.log(2)) < 1e-15


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    w = mlp.compute_weights(mlp.init_params(3))
    w["b1"] = rng.standard_normal(128) * 0.1
    w["b2"] = rng.standard_normal(128) * 0.1
    w["b3"] = rng.standard_normal(6) * 0.1
    x, s2, bits, _ = _awgn(16, 8.0, 4)
    _, g = mlp.loss_and_grad(w, x, s2, bits)
    h = 1e-6
    for name, _ in mlp.SHAPES:
        flat = w[name].ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.loss_and_grad(w, x, s2, bits)
            flat[idx] = old - h
            lm, _ = mlp.loss_and_grad(w, x, s2, bits)
            flat[idx] = old
            num = (lp - lm) / (2 * h)
            ana = g[name].ravel()[idx]
            assert abs(num - ana) <= 1e-6 * max(1.0, abs(ana)), (name, idx, num, ana)


def test_adam_steps_in_closed_form():
    """With a constant gradient the bias-corrected moments are g and g^2,
    so every step moves each parameter by lr * g / (|g| + eps)."""
    opt = mlp.Adam(lr=1e-3)
    th = np.array([0.5, -1.0, 2.0])
    g = np.array([3.0, -0.25, 1e-4])
    want = th.copy()
    for _ in range(3):
        th = opt.step(th, g)
        want = want - 1e-3 * g / (np.abs(g) + 1e-8)
        assert np.max(np.abs(th - want)) < 1e-12


@pytest.mark.parametrize("esn0", [12.0])
def test_training_approaches_the_exact_demapper(esn0):
    """A short training run on AWGN 4D-64 symbols: the loss falls by far
    more than an order of magnitude and the GMI comes within 0.4 bit of the
    exact log-sum-exp demapper's (never above it beyond sampling noise)."""
    x, s2, bits, _ = _awgn(1 << 14, esn0, 2)
    xt, s2t, bt, zt = _awgn(1 << 13, esn0, 3)
    th, losses = mlp.train(mlp.init_params(5), x, s2, bits, batch=512, steps=300, lr=3e-3, seed=0)
    assert np.mean(losses[-20:]) < losses[0] / 50
    g_mlp = chain.count(mlp.llr(mlp.compute_weights(th), xt, s2t), bt.astype(float))["gmi"]
    g_ex = chain.count(chain.llr(zt, s2t[0], oracle_format("gs4d64")), bt.astype(float))["gmi"]
    assert g_ex - 0.4 < g_mlp < g_ex + 0.01
