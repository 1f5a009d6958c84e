"""Parity at the launch shape of the throughput benchmark.

The benchmark runs nine 4D-64 streams (Es/N0 8 .. 16 dB, 1000 km, FFT 4096 /
overlap 1024, 31 taps, 64 test phases, window 64) through one handle in
blocks of 2^16 symbols with tap lag 3 (Sec. 2: the adaptation of one buffer
serves later buffers, beside the parallel kernels).  At that size every
kernel runs the grids the benchmark times: the phase search takes ~67
32-symbol chunks per block (its 10-chunk shared ring wraps many times), the
range split and the ticketed partial sums of the fused de-rotation/demap
span ~30 blocks per stream, and the LMS of block n runs on the side stream
beside blocks n+1 and n+2.  Here the same handle settings run 2^18 symbols
per stream (four blocks, so block 3 uses the first adapted taps) against the
FP64 oracle under the near-tie protocol of the other end-to-end tests, the
slip-prone 8 dB stream included, and the phase-search stage runs alone on
nine streams of one 2^16-symbol block.
"""
import numpy as np
import pytest

from oracle import oracle_format

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pp = pytest.importorskip("parity_protocol")
jobs = pytest.importorskip("oracle_jobs")

FMT = "gs4d64"
N = 1 << 18
ESN0 = list(range(8, 17))
PARAMS = dict(cd_ps_per_nm=17000.0, n_fft=4096, n_ov=1024, taps=31, bps_phases=64, bps_window=64,
              block=1 << 16, n_upd=1024, lag=3, mu=1e-3, n_pre=2048, cma_passes=1, n_cma=0,
              n_train=1024, train_passes=3, skip_head=16384, skip_tail=512)
RX_KEYS = dict(fft=4096, overlap=1024, bps_window=64, block=1 << 16, n_upd=1024, lag=3, mu=1e-3,
               n_pre=2048, cma_passes=1, n_cma=0, n_train=1024, train_passes=3, skip_head=16384,
               skip_tail=512)


@pytest.fixture(scope="module")
def oracle_runs():
    from paper_2108_07004_gb300 import synth
    js = [dict(fmt=FMT, n_sym=N, seed=synth.stream_seed(2, 100 + i), esn0_db=float(e),
               cd_ps_per_nm=17000.0, linewidth_ts=2e-5, params=PARAMS, valid=True) for i, e in enumerate(ESN0)]
    return jobs.run_jobs(js)


def _receiver(S):
    from paper_2108_07004_gb300 import rx
    return rx.Receiver(FMT, cd_ps_per_nm=17000.0, taps=31, bps_phases=64, streams=S, **RX_KEYS)


def _state(rx, ress, p, fmt, n, counters):
    """The oracle's block-n state of every stream, in one state buffer."""
    from oracle import chain
    S = len(ress)
    stts = [chain.state_at(res, p, n) for res in ress]
    L = p.lag
    taps = np.stack([np.stack([stt["taps"][j] for stt in stts]) for j in range(L)])
    carry = np.array([stt["carry"] for stt in stts])
    y_tail = np.stack([stt["y_tail"] for stt in stts])
    u = {stt["lms_updates"] for stt in stts}
    assert len(u) == 1
    hd = dict(streams=S, taps=p.taps, lag=L, bps_window=p.bps_window, bps_phases=p.bps_phases,
              m_bits=fmt.m, block=p.block, n_sym=N, blocks_done=n, lms_updates=u.pop())
    return rx.pack_state(hd, taps, carry, y_tail, counters)


def _resume_points(res, p):
    """Blocks from which a near-tie in an earlier LMS span may have changed
    the taps (block nb's tie reaches block nb + lag)."""
    tie = res.bps_gap < pp.TIE
    dd_ties = {k for k, mg in res.dd_margin if mg < pp.DD_TIE}
    nblk = len(res.ranges)
    out = set()
    for nb in range(nblk):
        span = range(nb * p.block, min(nb * p.block + p.n_upd, N))
        if any(tie[k] or k in dd_ties for k in span) and nb + p.lag < nblk:
            out.add(nb + p.lag)
    return out


def test_chain_at_bench_launch_shape(oracle_runs):
    _chain_check(oracle_runs, bps_tc=0)


def _chain_check(oracle_runs, bps_tc, sm_reserve=0):
    from oracle import chain
    from paper_2108_07004_gb300 import rx
    fmt = oracle_format(FMT)
    p = chain.RxParams(**PARAMS)
    S = len(oracle_runs)
    sts = [o[0] for o in oracle_runs]
    ress = [o[1] for o in oracle_runs]
    nblk = len(ress[0].ranges)
    assert nblk == 4
    r = _receiver(S)
    r.set("bps_tc", bps_tc)
    r.set("sm_reserve", sm_reserve)
    r.set_reference(torch.from_numpy(np.stack([st.bits for st in sts])).cuda())
    samples = torch.from_numpy(np.stack([st.rx for st in sts])).cuda()
    llr = torch.zeros((S, N, fmt.m), dtype=torch.float32, device="cuda")
    cuts = sorted(set().union(*[_resume_points(res, p) for res in ress]))
    bounds = [0] + cuts + [nblk]
    for n0, n1 in zip(bounds[:-1], bounds[1:]):
        if n0 > 0:
            counters = rx.unpack_state(r.get_state())["counters"]
            r.set_state(_state(rx, ress, p, fmt, n0, counters))
        _, stats = r.process_blocks(samples, n0, n1, llr)
    g_all = llr.cpu().numpy().astype(np.float64)
    c0, c1 = p.skip_head, N - p.skip_tail
    for s in range(S):
        res, g, ref = ress[s], g_all[s], ress[s].llr
        fails = []
        amb = np.abs(ref) < 1e-4
        for n, (a, e) in enumerate(res.ranges):
            L0, dL, t_range, env = oracle_runs[s][2][n]
            fails += pp.check_block(g[a:e], L0, dL, t_range, env, a)
            t_max = max(abs(t_range[0]), abs(t_range[1]))
            amb[a:e] |= np.abs(L0) <= 1e-4 + np.abs(dL) * t_max
            for k, (lo, hi) in env.items():
                amb[k] |= (lo <= 1e-4) & (hi >= -1e-4)
        assert not fails, f"stream {s} ({ESN0[s]} dB), resumes at {cuts}: {len(fails)} rows fail: {fails[:6]}"
        assert (((g < 0) != (ref < 0)) & ~amb).sum() == 0, s
        mine = int(np.sum((g[c0:c1] < 0).astype(np.uint8) != sts[s].bits[c0:c1]))
        assert stats[s]["bit_errors"] == mine, s
        if not (res.bps_gap[c0:c1] < pp.TIE).any():
            assert stats[s]["bit_errors"] == res.stats["bit_errors"], s
            assert abs(stats[s]["gmi"] - res.stats["gmi"]) < 1e-4 * fmt.m, s


def test_phase_search_stage_nine_streams_one_block(oracle_runs):
    """rx_bps on the oracle's equaliser output of block 1 of all nine
    streams (range [block - W/2, 2 block - W/2), windows truncated at
    2 block, as in the chain): every CTA covers dozens of chunks, so the
    shared chunk ring wraps; indices equal the oracle's outside near-ties."""
    from oracle import chain
    p = chain.RxParams(**PARAMS)
    S = len(oracle_runs)
    ress = [o[1] for o in oracle_runs]
    a, e, nv = p.block - p.bps_window // 2, 2 * p.block - p.bps_window // 2, 2 * p.block
    assert ress[0].ranges[1] == (a, e)
    y = np.stack([res.y[:, :nv] for res in ress]).astype(np.complex64)
    r = _receiver(S)
    bo = torch.zeros((S, e - a), dtype=torch.uint8, device="cuda")
    r.bps(torch.from_numpy(y).cuda(), a, e, nv, bo)
    g = bo.cpu().numpy().astype(np.int64)
    for s, res in enumerate(ress):
        diff = g[s] != res.b[a:e]
        assert np.all(res.bps_gap[a:e][diff] < pp.TIE), (s, int(diff.sum()))
        assert diff.mean() < 1e-3, s


def test_phase_search_tensor_cores_nine_streams_one_block(oracle_runs):
    """The same stage on the tensor cores (bps_tc = 1: the orbit correlations
    as a tcgen05 TF32 product with a high/low split, SIMT epilogue): indices
    equal the oracle's outside near-ties."""
    from oracle import chain
    from paper_2108_07004_gb300 import rx
    p = chain.RxParams(**PARAMS)
    S = len(oracle_runs)
    ress = [o[1] for o in oracle_runs]
    a, e, nv = p.block - p.bps_window // 2, 2 * p.block - p.bps_window // 2, 2 * p.block
    y = np.stack([res.y[:, :nv] for res in ress]).astype(np.complex64)
    r = _receiver(S)
    r.set("bps_tc", 1)
    assert r.get("bps_tc") == 1
    bo = torch.zeros((S, e - a), dtype=torch.uint8, device="cuda")
    r.bps(torch.from_numpy(y).cuda(), a, e, nv, bo)
    g = bo.cpu().numpy().astype(np.int64)
    for s, res in enumerate(ress):
        diff = g[s] != res.b[a:e]
        assert np.all(res.bps_gap[a:e][diff] < pp.TIE), (s, int(diff.sum()))
        assert diff.mean() < 1e-3, s


def test_chain_at_bench_launch_shape_tensor_cores(oracle_runs):
    """The whole chain at the bench's launch shape with the phase search on
    the tensor cores, under the same protocol as the SIMT chain."""
    _chain_check(oracle_runs, bps_tc=1)


def test_chain_at_bench_launch_shape_frames_in_flight_grids(oracle_runs):
    """The grids the bench's handles use with two frames in flight (18 SMs
    left to the other frame: fewer, longer phase-search ranges per stream,
    another split of the blocks' sigma^2 sums), under the same protocol."""
    _chain_check(oracle_runs, bps_tc=0, sm_reserve=18)
