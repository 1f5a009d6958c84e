"""Serving with continuous batching (rx_server_*): every request's LLRs and
counts are the same alone and in a mix of requests of different formats,
lengths and links — in every issue mode, with several blocks per step, with
block latency timed, from several host threads and through the server's own
loop — and a small device-memory budget makes requests queue without
changing any result."""
import numpy as np
import pytest

from paper_2108_07004_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (format, symbols, km, Es/N0 dB, taps, B)
REQS = [("dp_qpsk", 20000, 80, 12.0, 15, 32), ("gs4d64", 50000, 1000, 14.0, 31, 64),
        ("dp_16qam", 33000, 300, 18.0, 15, 32), ("gs4d64", 70001, 2000, 14.0, 31, 64),
        ("dp_qpsk", 45000, 1500, 12.0, 31, 32), ("dp_16qam", 18000, 80, 18.0, 15, 32)]
M = {"dp_qpsk": 4, "dp_16qam": 8, "gs4d64": 6}


@pytest.fixture(scope="module")
def streams():
    out = []
    for i, (fmt, n, km, esn0, T, B) in enumerate(REQS):
        st = synth.make_stream(fmt, n, seed=synth.stream_seed(5, i), esn0_db=esn0,
                               cd_ps_per_nm=17.0 * km, linewidth_ts=1e-5)
        out.append((torch.from_numpy(st.rx.astype(np.complex64)).cuda(),
                    torch.from_numpy(st.bits).cuda()))
    return out


def _submit(srv, i, samples, bits):
    fmt, n, km, esn0, T, B = REQS[i]
    llr = torch.full((n, M[fmt]), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()                 # the fill is done before the request's stream writes
    rid = srv.submit(fmt, samples, llr, bits, cd_ps_per_nm=17.0 * km, taps=T, bps_phases=B,
                     fft=4096, overlap=1024, block=16384, n_pre=2048)
    return rid, llr


def _serve(idx, streams, budget=1 << 33, slots=16, issue=None, blocks_per_step=None):
    from paper_2108_07004_gb300 import rx
    srv = rx.Server(budget, slots)
    if issue is not None:
        srv.set_param("issue", issue)
    if blocks_per_step is not None:
        srv.set_param("blocks_per_step", blocks_per_step)
    got = {i: _submit(srv, i, *streams[i]) for i in idx}
    srv.run()
    torch.cuda.synchronize()
    res = {}
    for i, (rid, llr) in got.items():
        state, stats = srv.poll(rid)
        assert state == rx.REQ_DONE
        res[i] = (llr.cpu().numpy(), stats)
    info = srv.info()
    srv.close()
    return res, info


def test_each_result_is_the_same_alone_and_in_the_mix(streams):
    alone = {i: _serve([i], streams)[0][i] for i in range(len(REQS))}
    mix, info = _serve(range(len(REQS)), streams)
    assert info["max_active"] == len(REQS)
    for i in range(len(REQS)):
        assert np.array_equal(alone[i][0], mix[i][0]), i
        assert not np.isnan(mix[i][0]).any()
        for k in ("bit_errors", "n_sym", "gmi_sum"):
            assert alone[i][1][k] == mix[i][1][k], (i, k)


@pytest.mark.parametrize("issue", [0, 1, 2])
def test_issue_modes_give_the_results_of_the_multi_stream_handle(streams, issue):
    """The handles' issue modes (0: stages on their own streams with events;
    1: every launch on the request's stream; 2: blocks after the first as
    CUDA graphs updated in place) serve every request of the mix with the
    LLRs and counts of the request alone in mode 0."""
    alone = {i: _serve([i], streams, issue=0)[0][i] for i in range(len(REQS))}
    mix, info = _serve(range(len(REQS)), streams, issue=issue)
    assert info["max_active"] == len(REQS)
    for i in range(len(REQS)):
        assert np.array_equal(alone[i][0], mix[i][0]), (issue, i)
        for k in ("bit_errors", "n_sym", "gmi_sum"):
            assert alone[i][1][k] == mix[i][1][k], (issue, i, k)


@pytest.mark.parametrize("issue,bps", [(1, 3), (1, 1 << 20), (0, 2), (2, 3)])
def test_several_blocks_per_step_give_the_same_results(streams, issue, bps):
    """Issuing several blocks of a request per step (one rx_process_blocks
    call over them, the whole request for 2^20) changes no LLR and no count
    of any request of the mix, in each issue mode."""
    alone = {i: _serve([i], streams, issue=0)[0][i] for i in range(len(REQS))}
    mix, info = _serve(range(len(REQS)), streams, issue=issue, blocks_per_step=bps)
    assert info["max_active"] == len(REQS)
    for i in range(len(REQS)):
        assert np.array_equal(alone[i][0], mix[i][0]), (issue, bps, i)
        for k in ("bit_errors", "n_sym", "gmi_sum"):
            assert alone[i][1][k] == mix[i][1][k], (issue, bps, i, k)


def test_block_latency_times_every_issue_call(streams):
    """With "block_latency" on, every issue call of every request is timed
    (one time per call of blocks_per_step blocks, all positive) and the
    results are those of the requests alone."""
    from paper_2108_07004_gb300 import rx
    alone = {i: _serve([i], streams)[0][i] for i in range(len(REQS))}
    srv = rx.Server(1 << 33, 16)
    srv.set_param("blocks_per_step", 2)
    srv.set_param("block_latency", 1)
    got = {i: _submit(srv, i, *streams[i]) for i in range(len(REQS))}
    srv.run()
    torch.cuda.synchronize()
    srv.step()                               # retires what the last step left running
    for i, (rid, llr) in got.items():
        state, stats = srv.poll(rid)
        assert state == rx.REQ_DONE
        assert np.array_equal(llr.cpu().numpy(), alone[i][0]), i
    lat = srv.block_latency()
    calls = sum(-(-(-(-n // 16384)) // 2) for _, n, *_ in REQS)    # ceil(ceil(n / block) / 2)
    assert len(lat) == calls and min(lat) > 0.0, (len(lat), calls)
    srv.set_param("block_latency", 1)        # turning it on again clears the times
    assert srv.block_latency() == []
    srv.close()


def test_server_loop_admits_requests_submitted_while_it_runs(streams):
    """The server's own loop (rx_server_start): requests submitted one by one
    while it runs are admitted and issued without step() calls, each with
    the result of the request alone; step() is refused while the loop runs,
    and after stop() the caller steps again."""
    import time
    from paper_2108_07004_gb300 import rx
    alone = {i: _serve([i], streams)[0][i] for i in range(len(REQS))}
    srv = rx.Server(1 << 33, 16)
    srv.start()
    assert srv.get_param("running") == 1
    with pytest.raises(rx.RxError):
        srv.step()
    with pytest.raises(rx.RxError):
        srv.start()
    got = {}
    for i in range(len(REQS)):
        got[i] = _submit(srv, i, *streams[i])
        time.sleep(0.002)
    t0 = time.time()
    while any(srv.poll(rid)[0] not in (rx.REQ_DONE, rx.REQ_FAILED) for rid, _ in got.values()):
        assert time.time() - t0 < 60.0, "requests not finished by the server's loop"
        time.sleep(0.001)
    torch.cuda.synchronize()
    for i, (rid, llr) in got.items():
        state, stats = srv.poll(rid)
        assert state == rx.REQ_DONE
        assert np.array_equal(llr.cpu().numpy(), alone[i][0]), i
        assert stats["bit_errors"] == alone[i][1]["bit_errors"]
    srv.stop()
    assert srv.get_param("running") == 0
    rid, llr = _submit(srv, 0, *streams[0])  # stepped by the caller again
    srv.run()
    torch.cuda.synchronize()
    assert srv.poll(rid)[0] == rx.REQ_DONE
    assert np.array_equal(llr.cpu().numpy(), alone[0][0])
    srv.close()


def test_pooled_handle_grows_for_a_longer_request(streams):
    """A request longer than the pooled handle it reuses (same key) grows
    that handle's buffers: the server counts one regrow, creates no second
    handle, and the result is that of the request served alone."""
    from paper_2108_07004_gb300 import rx
    i_short, i_long = 1, 3                  # gs4d64, 50000 then 70001 symbols, 31 taps, B = 64
    alone = _serve([i_long], streams)[0][i_long]
    srv = rx.Server(1 << 33, 4)
    _submit(srv, i_short, *streams[i_short])
    srv.run()
    rid, llr = _submit(srv, i_long, *streams[i_long])
    srv.run()
    torch.cuda.synchronize()
    state, stats = srv.poll(rid)
    assert state == rx.REQ_DONE
    assert (srv.get_param("handles_created"), srv.get_param("handle_regrows"),
            srv.get_param("handles_destroyed")) == (1, 1, 0)
    srv.close()
    assert np.array_equal(llr.cpu().numpy(), alone[0])
    assert stats["bit_errors"] == alone[1]["bit_errors"]


def test_graph_issue_block_by_block_equals_one_call(streams):
    """A handle in issue mode 2 fed block by block (the first call direct,
    the others as one instantiated graph updated per block) gives the LLRs
    and counts of one rx_process call in mode 0."""
    from paper_2108_07004_gb300 import rx
    i = 3
    fmt, n, km, esn0, T, B = REQS[i]
    samples, bits = streams[i]
    kw = dict(cd_ps_per_nm=17.0 * km, taps=T, bps_phases=B, fft=4096, overlap=1024, block=8192, n_pre=2048)
    r0 = rx.Receiver(fmt, **kw)
    r0.set_reference(bits[None].contiguous())
    ref, st0 = r0.process(samples[None].contiguous())
    r2 = rx.Receiver(fmt, **kw)
    r2.set("issue", 2)
    r2.set_reference(bits[None].contiguous())
    nblk = (n + 8191) // 8192
    llr = torch.full_like(ref, float("nan"))
    for b in range(nblk):
        _, st2 = r2.process_blocks(samples[None].contiguous(), b, b + 1, llr, stats=b == nblk - 1)
    torch.cuda.synchronize()
    assert np.array_equal(llr.cpu().numpy(), ref.cpu().numpy())
    assert st2[0]["bit_errors"] == st0[0]["bit_errors"] and st2[0]["gmi_sum"] == st0[0]["gmi_sum"]


def test_served_request_equals_a_handle(streams):
    from paper_2108_07004_gb300 import rx
    i = 1
    fmt, n, km, esn0, T, B = REQS[i]
    samples, bits = streams[i]
    r = rx.Receiver(fmt, cd_ps_per_nm=17.0 * km, taps=T, bps_phases=B, fft=4096, overlap=1024,
                    block=16384, n_pre=2048)
    r.set_reference(bits[None].contiguous())
    ref, st = r.process(samples[None].contiguous())
    served, _ = _serve([i], streams)
    assert np.array_equal(served[i][0], ref[0].cpu().numpy())
    assert served[i][1]["bit_errors"] == st[0]["bit_errors"]


def test_small_budget_queues_without_changing_results(streams):
    alone = {i: _serve([i], streams)[0][i] for i in range(len(REQS))}
    # room for about two of the requests at a time
    budget = 53 * 2 * 70001 + 3 * (1 << 20)
    mix, info = _serve(range(len(REQS)), streams, budget=budget)
    assert 1 <= info["max_active"] <= 3
    assert info["mem_used"] == 0
    for i in range(len(REQS)):
        assert np.array_equal(alone[i][0], mix[i][0]), i


def test_request_larger_than_the_budget_is_refused(streams):
    from paper_2108_07004_gb300 import rx
    srv = rx.Server(1 << 20, 4)
    with pytest.raises(rx.RxError):
        _submit(srv, 1, *streams[1])
    srv.close()


def test_many_concurrent_requests_issued_from_several_threads(streams):
    """Four copies of every request at once (24 running): a step's blocks are
    issued from several host threads, with first launches of different
    formats and test-phase counts (different shared-memory sizes) racing;
    every copy must finish with the result of the request served alone."""
    from paper_2108_07004_gb300 import rx
    alone = {i: _serve([i], streams)[0][i] for i in range(len(REQS))}
    srv = rx.Server(1 << 34, 64)
    got = [(i, _submit(srv, i, *streams[i])) for _ in range(4) for i in range(len(REQS))]
    srv.run()
    torch.cuda.synchronize()
    for i, (rid, llr) in got:
        state, stats = srv.poll(rid)
        assert state == rx.REQ_DONE, (i, rx.lib().rx_server_last_error().decode())
        assert np.array_equal(llr.cpu().numpy(), alone[i][0]), i
        assert stats["bit_errors"] == alone[i][1]["bit_errors"]
    assert srv.info()["max_active"] == 4 * len(REQS)
    srv.close()


def test_reused_handle_without_reference_forgets_the_previous_one(streams):
    """A request without reference bits that reuses a pooled handle (same
    format, rate, taps and test phases) after a longer request with
    reference bits: no training stage and no counting, exactly as when it
    is served alone on a fresh server."""
    from paper_2108_07004_gb300 import rx
    i_long, i_short = 3, 1                  # gs4d64, 70001 and 50000 symbols, 31 taps, B = 64
    fmt, n, km, esn0, T, B = REQS[i_short]
    samples, _ = streams[i_short]

    def submit_plain(srv):
        llr = torch.full((n, M[fmt]), float("nan"), dtype=torch.float32, device="cuda")
        rid = srv.submit(fmt, samples, llr, None, cd_ps_per_nm=17.0 * km, taps=T, bps_phases=B,
                         fft=4096, overlap=1024, block=16384, n_pre=2048)
        return rid, llr

    alone = rx.Server(1 << 33, 4)
    rid_a, llr_a = submit_plain(alone)
    alone.run()
    torch.cuda.synchronize()
    _, stats_a = alone.poll(rid_a)
    alone.close()

    srv = rx.Server(1 << 33, 4)
    _submit(srv, i_long, *streams[i_long])  # with reference bits: trains and counts
    srv.run()
    rid, llr = submit_plain(srv)            # takes over that request's pooled handle
    srv.run()
    torch.cuda.synchronize()
    state, stats = srv.poll(rid)
    srv.close()
    assert state == rx.REQ_DONE
    assert stats_a["n_sym"] == 0 and stats["n_sym"] == 0 and stats["bit_errors"] == 0
    assert np.array_equal(llr.cpu().numpy(), llr_a.cpu().numpy())


def test_issue_settings_are_validated(streams):
    """The handle's "issue" takes 0, 1 or 2 and "fir_tma" 0 or 1; the
    server's "issue" the same and "issue_threads" 1 .. 64; anything else is
    refused."""
    from paper_2108_07004_gb300 import rx
    r = rx.Receiver("dp_qpsk", cd_ps_per_nm=1360.0, taps=15, bps_phases=32)
    for key, good, bad in (("issue", (0, 1, 2), (3, -1, 0.5)), ("fir_tma", (0, 1), (2,))):
        for v in good:
            r.set(key, v)
            assert r.get(key) == v
        for v in bad:
            with pytest.raises(rx.RxError):
                r.set(key, v)
    srv = rx.Server(1 << 30, 4)
    srv.set_param("issue", 2)
    srv.set_param("issue_threads", 3)
    for key, v in (("issue", 5), ("issue_threads", 0), ("issue_threads", 65), ("nothing", 1)):
        with pytest.raises(rx.RxError):
            srv.set_param(key, v)
    srv.close()
