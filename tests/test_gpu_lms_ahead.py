"""DD-LMS decisions taken a sub-block ahead change nothing.

Each DD update's decision is taken at the start of its 16-update sub-block on
the update's partial output p_k, with the margin T_k between the nearest and
the second-nearest table point; the update keeps that point while
2 |y_k - p_k| stays below T_k minus a slack, else it runs the warp-wide
nearest-point search on y_k (parameter lms_exact = 1 runs that search on
every update).  By the triangle inequality no other point can then be nearer
to y_k, so the decisions, and with one fixed rounding of the error on both
paths the taps, are those of the search on every update: the whole chain's
LLRs and counters must agree bit for bit, at the benchmark's launch shape
(nine 4D-64 streams, 8 .. 16 dB, where some updates fall back) and for the
2D tables (per-polarisation decisions, one orbit for QPSK, four and sixteen
for 16QAM and 64QAM).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = dict(bps_window=64, block=1 << 16, n_upd=1024, lag=3, mu=1e-3, n_pre=2048, cma_passes=1, n_cma=0,
            n_train=1024, train_passes=3, skip_head=16384, skip_tail=512)


def _streams(fmt, n, esn0, cd, seed0):
    from paper_2108_07004_gb300 import synth
    rxs, bits = [], []
    for i, e in enumerate(esn0):
        st = synth.make_stream(fmt, n, seed=synth.stream_seed(7, seed0 + i), esn0_db=float(e),
                               cd_ps_per_nm=cd, linewidth_ts=2e-5)
        rxs.append(st.rx)
        bits.append(st.bits)
    return np.stack(rxs), np.stack(bits)


def _run(fmt, samples, bits, exact, cd, taps, phases, **keys):
    from paper_2108_07004_gb300 import rx
    S, n = samples.shape[0], bits.shape[1]
    r = rx.Receiver(fmt, cd_ps_per_nm=cd, taps=taps, bps_phases=phases, streams=S, **keys)
    r.set("lms_exact", exact)
    assert r.get("lms_exact") == exact
    r.set_reference(torch.from_numpy(bits).cuda())
    llr = torch.empty((S, n, bits.shape[2]), dtype=torch.float32, device="cuda")
    r.process(torch.from_numpy(samples).cuda(), llr, stats=True)
    torch.cuda.synchronize()
    st = r.stats()
    r.close()
    return llr.cpu().numpy(), st


def _same(fmt, esn0, cd, taps, phases, n, seed0, **keys):
    samples, bits = _streams(fmt, n, esn0, cd, seed0)
    a, sa = _run(fmt, samples, bits, 0, cd, taps, phases, **keys)
    b, sb = _run(fmt, samples, bits, 1, cd, taps, phases, **keys)
    assert np.isfinite(a).all()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert sa == sb
    return sa


def test_ahead_equals_exact_search_bench_shape():
    st = _same("gs4d64", list(range(8, 17)), 17000.0, 31, 64, 1 << 18, 0, fft=4096, overlap=1024, **KEYS)
    assert sum(s["n_sym"] for s in st) > 0


@pytest.mark.parametrize("fmt,esn0", [("dp_qpsk", [9.0, 12.0]), ("dp_16qam", [15.0, 18.0]),
                                      ("dp_64qam", [21.0, 24.0]), ("gs128", [18.0, 20.0])])
def test_ahead_equals_exact_search_2d(fmt, esn0):
    """GS-128 (32 orbits per polarisation): the exact search spreads the
    orbits over all 32 lanes, the decisions taken ahead search 16 then the
    rest serially."""
    phases = 64 if fmt in ("dp_64qam", "gs128") else 32
    _same(fmt, esn0, 1360.0, 15, phases, 1 << 17, 20, fft=1024, overlap=256, **KEYS)
