"""Block-range processing and checkpoint / resume of the stream state
(rx_process_blocks, rx_get_state, rx_set_state) through the C ABI.

The chain is deterministic (fixed-order reductions), so a stream processed
in pieces, or resumed in another handle from a saved state, must give the
same bytes as one rx_process over it."""
import numpy as np
import pytest

from paper_2108_07004_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 20000          # five blocks of 4096, the last one ragged


@pytest.fixture(scope="module")
def stream():
    st = synth.make_stream("dp_16qam", N, seed=synth.stream_seed(9, 7), esn0_db=17.0,
                           cd_ps_per_nm=1000.0, linewidth_ts=1e-5)
    return torch.from_numpy(st.rx[None].astype(np.complex64)).cuda(), \
        torch.from_numpy(st.bits[None]).cuda()


def _receiver(lag, bits):
    from paper_2108_07004_gb300 import rx
    r = rx.Receiver("dp_16qam", cd_ps_per_nm=1000.0, taps=15, bps_phases=32)
    r.set("block", 4096)
    r.set("lag", lag)
    r.set("n_pre", 4096)
    r.set("n_cma", 1500)            # the CMA -> DD switch falls inside block 1
    r.set_reference(bits)
    return r


def _same_stats(a, b):
    for k in ("n_sym", "bit_errors", "gmi_sum", "evm_num", "evm_den", "sigma2_last", "blocks"):
        assert a[k] == b[k], k


@pytest.mark.parametrize("lag", [1, 2])
def test_blocks_in_pieces_equal_one_call(stream, lag):
    x, bits = stream
    ref, st_ref = _receiver(lag, bits).process(x)
    r = _receiver(lag, bits)
    llr = torch.zeros_like(ref)
    for b0, b1 in ((0, 1), (1, 3), (3, 5)):
        _, st = r.process_blocks(x, b0, b1, llr)
    assert torch.equal(llr, ref)
    _same_stats(st[0], st_ref[0])


@pytest.mark.parametrize("lag", [1, 2])
def test_state_resumes_in_another_handle(stream, lag):
    from paper_2108_07004_gb300 import rx
    x, bits = stream
    ref, st_ref = _receiver(lag, bits).process(x)
    a = _receiver(lag, bits)
    la, _ = a.process_blocks(x, 0, 2)
    blob = a.get_state()
    s = rx.unpack_state(blob)
    assert (s["blocks_done"], s["n_sym"], s["lms_updates"], s["lag"]) == (2, N, 2 * 1024, lag)
    assert s["ring"].shape == (lag, 1, 2, 2, 15) and s["y_tail"].shape == (1, 2, 64)
    b = _receiver(lag, bits)
    b.set_state(blob)
    assert b.get_state() == blob                   # restored exactly
    lb, st = b.process_blocks(x, 2, 5)
    row = 2 * 4096 - 32                             # first row of block 2's range
    assert torch.equal(la[:, :row], ref[:, :row])
    assert torch.equal(lb[:, row:], ref[:, row:])
    _same_stats(st[0], st_ref[0])


def test_state_and_range_errors(stream):
    from paper_2108_07004_gb300 import rx
    x, bits = stream
    r = _receiver(1, bits)
    with pytest.raises(rx.RxError) as e:
        r.get_state()                               # nothing processed yet
    assert e.value.code == -6
    with pytest.raises(rx.RxError) as e:
        r.process_blocks(x, 2, 3)                   # does not continue a stream
    assert e.value.code == -6
    with pytest.raises(rx.RxError) as e:
        r.process_blocks(x, 0, 6)                   # beyond the 5 blocks
    assert e.value.code == -1
    r.process_blocks(x, 0, 2)
    blob = r.get_state()
    with pytest.raises(rx.RxError) as e:
        r.process_blocks(x, 3, 4)                   # skips block 2
    assert e.value.code == -6
    bad = bytearray(blob)
    bad[0] ^= 1                                     # magic
    for b_ in (bytes(bad), blob[:-8], blob + b"\0" * 8):
        with pytest.raises(rx.RxError) as e:
            r.set_state(b_)
        assert e.value.code == -1
    s = rx.unpack_state(blob)
    hd = {k: s[k] for k in rx.STATE_HEADER.names if k not in ("magic", "version")}
    for key, val in (("blocks_done", 0), ("blocks_done", 6), ("bps_phases", 64)):
        blob2 = rx.pack_state({**hd, key: val}, s["ring"], s["carry"], s["y_tail"], s["counters"])
        with pytest.raises(rx.RxError) as e:
            r.set_state(blob2)
        assert e.value.code == -1
    other = rx.Receiver("dp_16qam", cd_ps_per_nm=1000.0, taps=31, bps_phases=32)
    other.set("block", 4096)
    with pytest.raises(rx.RxError) as e:
        other.set_state(blob)                       # 15-tap state into a 31-tap handle
    assert e.value.code == -1
    # a rejected state changed nothing: the stream still continues at block 2
    r.process_blocks(x, 2, 3)


def test_builtin_gs4d64_equals_its_table_file():
    """RX_FMT_GS4D64 (the table compiled in from data/gs4d64_v1.json) gives
    the same receiver as the same table passed as a custom format."""
    from paper_2108_07004_gb300 import rx
    st = synth.make_stream("gs4d64", 20000, seed=synth.stream_seed(9, 77), esn0_db=13.0,
                           cd_ps_per_nm=2000.0, linewidth_ts=1e-5)
    out = []
    for fmt in ("gs4d64", "table:gs4d64"):
        r = rx.Receiver(fmt, cd_ps_per_nm=2000.0, taps=31, bps_phases=64, fft=4096, overlap=1024, block=4096)
        assert (r.dims, r.m, r.M) == (4, 6, 64)
        r.set_reference(torch.from_numpy(st.bits[None]).cuda())
        llr, stats = r.process(torch.from_numpy(st.rx[None]).cuda())
        out.append((llr.cpu().numpy(), stats[0]["bit_errors"]))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
