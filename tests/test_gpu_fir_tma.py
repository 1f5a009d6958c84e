"""The FIR with its input windows staged by the tensor memory accelerator
(parameter fir_tma = 1, the default) against the cp.async form (0): the same
bits for every storage kind, tap count, linear and widely-linear
butterflies, several streams, and output ranges that start at the stream's
first symbol (windows before sample 0, zero-filled by the copy), end at its
last (windows past the end), or sit inside it; where a row is not a whole
number of 64-byte groups (N not a multiple of 4 for float32, of 8 for
16-bit storage) the TMA form falls back to cp.async.  The TMA form is also held to the FP64 oracle's FIR (Sec. 2's
2x2 butterfly) directly."""
import numpy as np
import pytest

from oracle import chain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {0: None, 1: torch.float16, 2: torch.bfloat16}


def _rx():
    from paper_2108_07004_gb300 import rx
    return rx


def _store(z, prec):
    """complex64 [..., n] -> the storage of precision prec (bit-level tensor, last dim n)."""
    t = torch.from_numpy(np.ascontiguousarray(z.astype(np.complex64))).cuda()
    if prec == 0:
        return t
    f = torch.view_as_real(t).to(DT[prec]).contiguous()     # [..., n, 2]
    return f.view(torch.int32).squeeze(-1)


def _load(t, prec):
    if prec == 0:
        return t.cpu().numpy().astype(np.complex128)
    f = t.unsqueeze(-1).view(DT[prec]).float().cpu().numpy()
    return f[..., 0] + 1j * f[..., 1]


def _run(prec, T, wl, S, N, k0, k1, tma, x, taps):
    rx = _rx()
    r = rx.Receiver("dp_qpsk", cd_ps_per_nm=500.0, taps=T, bps_phases=32, streams=S)
    r.set("precision", prec)
    if wl:
        r.set("widely_linear", 1)
    r.set("fir_tma", tma)
    xs = _store(x, prec)
    n = k1 - k0
    y = torch.zeros((S, 2, n), dtype=torch.complex64 if prec == 0 else torch.int32, device="cuda")
    r.fir(xs, torch.from_numpy(taps.astype(np.complex64)).cuda(), k0, k1, y)
    torch.cuda.synchronize()
    return y


CASES = [
    # prec, T, wl, S, N, (k0, k1)
    (0, 31, 0, 1, 9000, (0, 9000)),
    (0, 31, 0, 3, 20000, (1000, 19993)),
    (0, 15, 0, 2, 6001, (0, 6001)),            # N not a multiple of 4: cp.async fallback
    (0, 7, 0, 1, 4096, (17, 4096)),
    (0, 31, 1, 2, 12000, (0, 12000)),
    (0, 15, 1, 1, 7000, (511, 6999)),
    (1, 31, 0, 2, 10000, (0, 10000)),
    (1, 15, 0, 1, 10001, (0, 10001)),          # N not a multiple of 8: cp.async fallback
    (1, 31, 1, 1, 8000, (100, 8000)),
    (2, 31, 0, 3, 12000, (0, 12000)),
    (2, 7, 0, 1, 5000, (3, 4990)),
    (2, 31, 1, 2, 9002, (0, 9002)),
]


@pytest.mark.parametrize("prec,T,wl,S,N,rng_", CASES)
def test_tma_fir_equals_cp_async_fir(prec, T, wl, S, N, rng_):
    k0, k1 = rng_
    g = np.random.default_rng(T * 1000 + N)
    x = (g.standard_normal((S, 2, 2 * N)) + 1j * g.standard_normal((S, 2, 2 * N))) * 0.5
    L = 2 * T if wl else T
    taps = 0.1 * (g.standard_normal((S, 2, 2, L)) + 1j * g.standard_normal((S, 2, 2, L)))
    a = _run(prec, T, wl, S, N, k0, k1, 1, x, taps)
    b = _run(prec, T, wl, S, N, k0, k1, 0, x, taps)
    assert torch.equal(a, b)
    assert not torch.isnan(a.float() if prec else a.abs()).any()


@pytest.mark.parametrize("T", [7, 15, 31])
def test_tma_fir_against_the_oracle(T):
    S, N = 2, 11000
    g = np.random.default_rng(T)
    x = ((g.standard_normal((S, 2, 2 * N)) + 1j * g.standard_normal((S, 2, 2 * N))) * 0.5).astype(np.complex64)
    taps = (0.1 * (g.standard_normal((S, 2, 2, T)) + 1j * g.standard_normal((S, 2, 2, T)))).astype(np.complex64)
    for k0, k1 in ((0, N), (4321, N - 5)):
        y = _run(0, T, 0, S, N, k0, k1, 1, x, taps)
        got = y.cpu().numpy()
        for s in range(S):
            ref = chain.fir(x[s].astype(np.complex128), taps[s].astype(np.complex128), k0, k1)
            rms = np.sqrt(np.mean(np.abs(ref) ** 2))
            assert np.max(np.abs(got[s] - ref)) < 1e-5 * rms, (T, s, k0)
