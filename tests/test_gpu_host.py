"""rx_process_host (host buffers, copies overlapped with the chain in groups
of blocks) gives exactly the LLRs and statistics of rx_process on device
buffers, with pinned and with pageable host memory."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rx():
    from paper_2108_07004_gb300 import rx
    return rx


@pytest.mark.parametrize("pinned", [True, False])
def test_process_host_equals_device_path(pinned):
    rx = _rx()
    from paper_2108_07004_gb300 import synth
    S, n = 3, 5 * 4096 + 1000                 # 6 blocks, the last one ragged: 3 groups
    sts = [synth.make_stream("dp_16qam", n, seed=synth.stream_seed(11, s), esn0_db=17.0,
                             cd_ps_per_nm=2000.0, linewidth_ts=1e-5) for s in range(S)]
    samples = np.stack([st.rx for st in sts]).astype(np.complex64)
    bits = np.stack([st.bits for st in sts])

    def receiver():
        r = rx.Receiver("dp_16qam", cd_ps_per_nm=2000.0, taps=15, bps_phases=32, streams=S)
        for k, v in (("fft", 1024), ("overlap", 256), ("block", 4096), ("n_pre", 4096), ("lag", 2)):
            r.set(k, v)
        r.set_reference(torch.from_numpy(bits).cuda())
        return r

    ref, st_ref = receiver().process(torch.from_numpy(samples).cuda())
    ref = ref.cpu()
    r = receiver()
    s_h = torch.from_numpy(samples)
    l_h = torch.full(tuple(ref.shape), float("nan"), dtype=torch.float32)
    if pinned:
        s_h, l_h = s_h.pin_memory(), l_h.pin_memory()
    st = r.process_host(s_h, l_h)
    assert torch.equal(l_h, ref)
    for a, b in zip(st, st_ref):
        assert a["bit_errors"] == b["bit_errors"] and a["n_sym"] == b["n_sym"]
        assert a["gmi"] == b["gmi"]
    # a second call on the same handle (a new stream through the same buffers)
    l2 = torch.zeros_like(l_h)
    r.reset()
    r.set_reference(torch.from_numpy(bits).cuda())
    r.process_host(s_h, l2, stats=False)
    assert torch.equal(l2, ref)


@pytest.mark.parametrize("n_train", [1024, 10000])
def test_host_reference_taken_in_by_groups(n_train):
    """rx_set_reference_host: the bits go in group by group inside
    rx_process_host (the training span with the first group); results equal
    those of a device reference, and a device entry point after it copies
    the pending reference whole."""
    rx = _rx()
    from paper_2108_07004_gb300 import synth
    S, n = 2, 5 * 4096 + 700
    sts = [synth.make_stream("dp_16qam", n, seed=synth.stream_seed(23, s), esn0_db=16.0,
                             cd_ps_per_nm=2000.0, linewidth_ts=1e-5) for s in range(S)]
    samples = np.stack([st.rx for st in sts]).astype(np.complex64)
    bits = np.stack([st.bits for st in sts])

    def receiver():
        r = rx.Receiver("dp_16qam", cd_ps_per_nm=2000.0, taps=15, bps_phases=32, streams=S)
        for k, v in (("fft", 1024), ("overlap", 256), ("block", 4096), ("n_pre", 4096), ("lag", 2),
                     ("n_train", n_train)):
            r.set(k, v)
        return r

    r0 = receiver()
    r0.set_reference(torch.from_numpy(bits).cuda())
    ref, st_ref = r0.process(torch.from_numpy(samples).cuda())
    ref = ref.cpu()
    assert st_ref[0]["n_sym"] > 0
    r = receiver()
    s_h = torch.from_numpy(samples).pin_memory()
    b_h = torch.from_numpy(bits).pin_memory()
    l_h = torch.full(tuple(ref.shape), float("nan"), dtype=torch.float32).pin_memory()
    r.set_reference_host(b_h)
    st = r.process_host(s_h, l_h)
    assert torch.equal(l_h, ref)
    for a, b in zip(st, st_ref):
        assert a["bit_errors"] == b["bit_errors"] and a["n_sym"] == b["n_sym"]
        assert a["gmi"] == b["gmi"]
    # pending host reference used by the device entry point
    r2 = receiver()
    r2.set_reference_host(b_h)
    l3, st3 = r2.process(torch.from_numpy(samples).cuda())
    assert torch.equal(l3.cpu(), ref)
    assert [a["bit_errors"] for a in st3] == [b["bit_errors"] for b in st_ref]
