"""The end-to-end acceptance rule of the GPU parity tests, checked on the
CPU with the oracle's own output and planted mistakes: it accepts every
result the near-tie choices allow (the oracle's LLRs; LLRs under another
valid block sigma^2; another valid phase at a near-tie symbol) and rejects
a block-wide scale error and a single wrong LLR beyond 1e-4 relative."""
import numpy as np
import pytest

from oracle import chain, oracle_format

gp = pytest.importorskip("test_gpu_parity")


@pytest.fixture(scope="module")
def qpsk():
    st, p, res = gp._oracle_run("qpsk80km")
    return p, res, oracle_format("dp_qpsk")


def test_accepts_valid_alternatives(qpsk):
    p, res, fmt = qpsk
    N = res.llr.shape[0]
    for n, (a, e) in enumerate(res.ranges):
        L0, dL, tr, env = gp._block_valid(res, p, fmt, n, N)
        assert env, "the case should have near-ties in every block"
        assert not gp._check_block(res.llr[a:e], L0, dL, tr, env, a)
        g = chain.llr(res.z[:, a:e], res.sigma2[n] + 0.7 * tr[1] + 0.3 * tr[0], fmt)
        for k, (lo, hi) in env.items():
            g[k - a] = lo if k % 2 else hi
        assert not gp._check_block(g, L0, dL, tr, env, a)


def test_rejects_planted_errors(qpsk):
    p, res, fmt = qpsk
    N = res.llr.shape[0]
    for n, (a, e) in enumerate(res.ranges):
        L0, dL, tr, env = gp._block_valid(res, p, fmt, n, N)
        width = tr[1] - tr[0]
        g = res.llr[a:e] * (1 + 2 * max(-tr[0], tr[1]) / res.sigma2[n] + 3e-4)
        assert gp._check_block(g, L0, dL, tr, env, a)
        g = res.llr[a:e].copy()
        i = (e - a) // 2
        while a + i in env:
            i += 1
        j = int(np.argmax(np.abs(g[i])))
        g[i, j] += np.sign(g[i, j]) * (3e-4 * max(1.0, abs(g[i, j])) + abs(dL[i, j]) * width)
        fails = gp._check_block(g, L0, dL, tr, env, a)
        assert [k for k, _ in fails] == [a + i]
        k = next(iter(env))
        g = res.llr[a:e].copy()
        g[k - a] = env[k][1] + 1e-3 * np.maximum(1.0, np.abs(env[k][1]))
        assert [kk for kk, _ in gp._check_block(g, L0, dL, tr, env, a)] == [k]
