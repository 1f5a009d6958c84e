"""GPU block LMS (groups of P updates sharing the taps at the group start)
against the FP64 oracle: the tap updates of one span in each mode, and the
whole chain with block updates against the oracle's chain (same segment
protocol as the exact chain)."""
import numpy as np
import pytest

from oracle import chain, oracle_format

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import test_gpu_parity as TP  # noqa: E402


@pytest.mark.parametrize("P", [4, 16, 64])
@pytest.mark.parametrize("case", ["qpsk80km", "gs1000km"])
def test_block_lms_span_parity(case, P):
    """CMA for the first 300 updates, DD after (the switch inside a group
    unless P divides 300), from the oracle's taps and phases of block 2."""
    st, p, res = TP._oracle_run(case)
    fmt = oracle_format(TP.CASES[case][0])
    x = res.x.astype(np.complex64)
    n = 2
    k0 = n * p.block
    h_in = res.taps_after[n - 1].astype(np.complex64)
    phase = {k: res.phi[k] for k in range(k0, k0 + p.n_upd)}
    p2 = chain.RxParams(**{**p.__dict__, "n_cma": 300})
    info = chain.LmsInfo()
    ref = chain.lms_block(x.astype(np.complex128), h_in.astype(np.complex128), range(k0, k0 + p.n_upd),
                          fmt, p2, P, u0=0, phase=phase, info=info)
    if min(mg for _, mg in info.dd_margin) <= 1e-4:
        pytest.skip("oracle has a near-tie decision in the span")
    pcode = (res.b.astype(np.int64) | ((res.m % fmt.sym_order) << 8)).astype(np.uint16)
    r = TP._receiver(case, lms_block=P, n_cma=300)
    taps = TP._dev(h_in[None])
    r.lms(TP._dev(x[None]), taps, k0, p.n_upd, TP._dev(pcode[None]), 2, 1, 0)
    g = taps[0].cpu().numpy()
    assert np.max(np.abs(g - ref)) < 2e-4 * np.max(np.abs(ref))
    # and it is not the sequential recursion
    seq = chain.lms(x.astype(np.complex128), h_in.astype(np.complex128), range(k0, k0 + p.n_upd), fmt, p2,
                    phase=phase)
    assert np.max(np.abs(seq - ref)) > 10 * np.max(np.abs(g - ref))


def test_block_lms_chain_end_to_end():
    """rx_process_blocks with groups of 16 against the oracle's chain with
    the same groups, 4D-64 over 1000 km, tap lag 2."""
    rx = TP._rx()
    case = "gs1000km"
    fmt_name, n, cd, nfft, nov, T, B, blk, esn0, lw = TP.CASES[case]
    from paper_2108_07004_gb300 import synth
    st = synth.make_stream(fmt_name, n, seed=synth.stream_seed(9, 77), esn0_db=esn0, cd_ps_per_nm=cd,
                           linewidth_ts=lw)
    p = chain.RxParams(**{**TP._params(case).__dict__, "lms_block": 16, "lag": 2})
    fmt = oracle_format(fmt_name)
    res = chain.run_chain(st.rx, fmt, p, ref_bits=st.bits)
    r = TP._receiver(case, lms_block=16, lag=2)
    r.set_reference(TP._dev(st.bits[None]))
    samples = TP._dev(st.rx[None])
    N = res.llr.shape[0]
    llr = torch.zeros((1, N, fmt.m), dtype=torch.float32, device="cuda")
    segs = TP._segments(res, p, N)
    for n0, n1 in segs:
        if n0 > 0:
            counters = rx.unpack_state(r.get_state())["counters"]
            r.set_state(TP._oracle_state(rx, res, p, fmt, n0, N, counters))
        r.process_blocks(samples, n0, n1, llr)
    g = llr[0].cpu().numpy().astype(np.float64)
    fails = []
    for nb, (a, e) in enumerate(res.ranges):
        L0, dL, t_range, env = TP._block_valid(res, p, fmt, nb, N)
        fails += TP._check_block(g[a:e], L0, dL, t_range, env, a)
    assert not fails, f"segments {segs}: {len(fails)} rows fail: {fails[:4]}"
