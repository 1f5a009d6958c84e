"""Streaming entry (rx_push / rx_flush): one continuous stream fed in ragged
buffers, as Sec. 2's real-time loop takes DMA buffers one after another.

Every push of n samples returns n/2 rows; row r of a stream holds symbol
r - d for the fixed delay d.  The rows after the delay plus the flushed rows
must equal, bit for bit, one rx_process over the whole stream (same kernels,
same block schedule), and so must the counters; the oracle comparison of the
streamed output follows the near-tie protocol of the other end-to-end tests.
"""
import math

import numpy as np
import pytest

from paper_2108_07004_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pp = pytest.importorskip("parity_protocol")

M = {"dp_qpsk": 4, "dp_16qam": 8, "gs4d64": 6}


def _delay_formula(block, fft, overlap, taps, W, n_pre, n_train):
    """The fixed delay as the header states it."""
    hop, D = fft - overlap, (taps - 1) // 2
    per = hop // math.gcd(2 * block, hop)
    k_st = max(n_pre, n_train)

    def need(n):
        return -(-(2 * max((n + 1) * block, k_st) + D) // hop) * hop + overlap // 2

    d = 0
    for n in range(per + -(-k_st // block) + 3):
        C = 0 if n == 0 else n * block - W // 2
        d = max(d, (need(n) - 1) // 2 - C)
    return d


def _receiver(fmt, S, cd, T, B, **kw):
    from paper_2108_07004_gb300 import rx
    return rx.Receiver(fmt, cd_ps_per_nm=cd, taps=T, bps_phases=B, streams=S, **kw)


def _streams(fmt, S, n, cd, esn0, seed0):
    sts = [synth.make_stream(fmt, n, seed=synth.stream_seed(7, seed0 + s), esn0_db=esn0, cd_ps_per_nm=cd,
                             linewidth_ts=1e-5) for s in range(S)]
    return np.stack([st.rx for st in sts]), np.stack([st.bits for st in sts])


def _pushed(r, samples, sizes):
    """Push samples [S, 2, 2N] in pieces of the given sizes, then flush;
    returns the stream's rows after the delay [S, N, m] and the per-call
    stats."""
    S, _, ns = samples.shape
    d = r.stream_delay()
    rows, firsts, c = [], [], 0
    for n in sizes:
        piece = samples[:, :, c:c + n].contiguous()
        llr, st = r.push(piece)
        assert llr.shape[1] == n // 2
        rows.append(llr.cpu().numpy())
        firsts.append((c // 2, n // 2, st[0]["first_valid"]))
        c += n
    assert c == ns
    llr, st_end = r.flush()
    N = ns // 2
    assert llr.shape[1] == min(N, d)
    rows.append(llr.cpu().numpy())
    out = np.concatenate(rows, axis=1)
    assert out.shape[1] == N + min(N, d)
    # the first d rows of the stream are the delay's zeros
    assert not out[:, : min(d, N)].any()
    for row0, cnt, fv in firsts:
        assert fv == min(cnt, max(0, d - row0))
    return out[:, min(d, N):], st_end


def _ragged_sizes(ns, seed, block):
    rng = np.random.default_rng(seed)
    sizes, c = [], 0
    choices = [0, 2, 2 * 61, 2 * 997, 2 * block - 2, 2 * block, 2 * 3 * block + 14, 2 * 5 * block + 6]
    while c < ns:
        n = int(rng.choice(choices)) if rng.random() < 0.5 else 2 * int(rng.integers(1, 3 * block))
        n = min(n, ns - c)
        sizes.append(n)
        c += n
    return sizes


CASES = {
    # name: (format, S, N, cd, Es/N0, taps, B, params)
    "gs4d64_lag3": ("gs4d64", 2, 77_777, 17000.0, 14.0, 31, 64,
                    dict(fft=4096, overlap=1024, block=4096, lag=3, n_pre=2048, skip_head=2048, skip_tail=300)),
    "qpsk_chains": ("dp_qpsk", 3, 50_001, 1360.0, 12.0, 15, 32,
                    dict(fft=1024, overlap=256, block=4096, lag=3, lms_start=1, skip_head=1024)),
    "qam16_half": ("dp_16qam", 2, 40_000, 2000.0, 18.0, 15, 32,
                   dict(fft=1024, overlap=256, block=2048, lag=2, precision=1)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_pushed_stream_equals_one_call(case):
    fmt, S, N, cd, esn0, T, B, kw = CASES[case]
    samples_np, bits_np = _streams(fmt, S, N, cd, esn0, 10 * list(CASES).index(case))
    samples = torch.from_numpy(samples_np).cuda()
    bits = torch.from_numpy(bits_np).cuda()
    whole = _receiver(fmt, S, cd, T, B, **kw)
    whole.set_reference(bits)
    ref, st_ref = whole.process(samples)
    ref = ref.cpu().numpy()
    r = _receiver(fmt, S, cd, T, B, **kw)
    d = r.stream_delay()
    assert d == _delay_formula(kw["block"], kw["fft"], kw["overlap"], T, 64, kw.get("n_pre", 2048), 1024)
    for seed in (1, 2):
        r.set_reference(bits)                   # before the stream's first push
        got, st = _pushed(r, samples, _ragged_sizes(2 * N, seed, kw["block"]))
        assert np.array_equal(got, ref), (seed, np.argwhere(got != ref)[:5])
        for s in range(S):
            for k in ("bit_errors", "n_sym", "gmi_sum", "evm_num", "blocks"):
                assert st[s][k] == st_ref[s][k], (seed, s, k)


def test_stream_shorter_than_the_delay():
    """A stream whose every symbol comes out of the flush."""
    fmt, S, N, cd, esn0, T, B, kw = CASES["gs4d64_lag3"]
    n = 5000                                    # d = 5919 at these settings
    samples_np, bits_np = _streams(fmt, S, n, cd, esn0, 77)
    samples = torch.from_numpy(samples_np).cuda()
    bits = torch.from_numpy(bits_np).cuda()
    whole = _receiver(fmt, S, cd, T, B, **kw)
    whole.set_reference(bits)
    ref, _ = whole.process(samples)
    r = _receiver(fmt, S, cd, T, B, **kw)
    assert r.stream_delay() > n
    r.set_reference(bits)
    got, _ = _pushed(r, samples, [2 * 1000, 2 * 3000, 0, 2 * 1000])
    assert np.array_equal(got, ref.cpu().numpy())


def test_pushed_stream_against_the_oracle():
    """The streamed rows of two parity cases against the FP64 oracle under the
    near-tie protocol: the blocks of the protocol's first segment (those the
    GPU and the oracle equalise with the same taps; a stream cannot be
    resumed from the oracle's state mid-push) are compared row by row, and
    the counts when that segment is the whole stream."""
    gp = pytest.importorskip("test_gpu_parity")
    from oracle import oracle_format
    compared = 0
    for case in ("gs1000km", "qpsk80km"):
        st, p, res = gp._oracle_run(case)
        N = res.llr.shape[0]
        n1 = pp.segments(res, p, N)[0][1]
        fmt = oracle_format(gp.CASES[case][0])
        r = gp._receiver(case)
        r.set_reference(torch.from_numpy(st.bits[None]).cuda())
        got, stats = _pushed(r, torch.from_numpy(st.rx[None]).cuda(), _ragged_sizes(2 * N, 5, p.block))
        g = got[0].astype(np.float64)
        fails = []
        for n in range(n1):
            a, e = res.ranges[n]
            L0, dL, t_range, env = pp.block_valid(res, p, fmt, n, N)
            fails += pp.check_block(g[a:e], L0, dL, t_range, env, a)
            compared += e - a
        assert not fails, (case, fails[:5])
        c0, c1 = p.skip_head, N - p.skip_tail
        assert stats[0]["bit_errors"] == int(np.sum((g[c0:c1] < 0).astype(np.uint8) != st.bits[c0:c1]))
    assert compared >= 4096


def test_stream_state_calls_and_errors():
    from paper_2108_07004_gb300 import rx
    fmt, S, N, cd, esn0, T, B, kw = CASES["qpsk_chains"]
    r = _receiver(fmt, S, cd, T, B, **kw)
    with pytest.raises(rx.RxError):
        r.flush()                                  # no stream
    x = torch.zeros((S, 2, 7), dtype=torch.complex64, device="cuda")
    with pytest.raises(rx.RxError):
        r.push(x)                                  # odd sample count
    _, st = r.push(torch.zeros((S, 2, 4096), dtype=torch.complex64, device="cuda"))
    assert st[0]["n_sym"] == 0 and st[0]["first_valid"] == 2048   # all delay rows so far
    with pytest.raises(rx.RxError):
        r.get_state()                              # streaming: no block state
    r.set("mu", 2e-3)                              # ends the stream without output
    with pytest.raises(rx.RxError):
        r.flush()


def test_bounded_wait():
    """rx_wait gives up with RX_ETIMEDOUT while the handle's stream is busy
    (a bounded spin of about 0.1 s queued on it) and succeeds once it is done."""
    fmt, S, N, cd, esn0, T, B, kw = CASES["qpsk_chains"]
    r = _receiver(fmt, S, cd, T, B, **kw)
    torch.cuda.synchronize()
    torch.cuda._sleep(200_000_000)                 # on the handle's (current) stream
    assert r.wait(0.0) is False
    assert r.wait(60_000.0) is True
