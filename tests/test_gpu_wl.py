"""GPU widely-linear butterfly (taps on x and conj(x), [S][2][2][2T])
against the FP64 oracle: the FIR, CMA and DD spans (sequential and block
LMS), the whole chain on a stream with a transmitter IQ imbalance, and the
gain over the linear butterfly there."""
import numpy as np
import pytest

from oracle import chain, oracle_format
from paper_2108_07004_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import test_gpu_parity as TP  # noqa: E402

IQ = (0.15, 0.12)        # gain error 15 %, phase error 0.12 rad
CASE = ("dp_16qam", 1 << 14, 1360.0, 1024, 256, 15, 32, 4096, 18.0, 1e-5)


def _wl(h, rng, scale=0.05):
    """linear taps [2,2,T] -> widely-linear [2,2,2T], conjugate taps random."""
    T = h.shape[2]
    g = scale * (rng.standard_normal((2, 2, T)) + 1j * rng.standard_normal((2, 2, T)))
    return np.concatenate([h, g], axis=2)


@pytest.mark.parametrize("case", ["qpsk80km", "gs1000km"])
def test_wl_fir_parity(case):
    st, p, res = TP._oracle_run(case)
    r = TP._receiver(case, widely_linear=1)
    x = res.x.astype(np.complex64)
    hw = _wl(res.w0, np.random.default_rng(3)).astype(np.complex64)
    k0, k1 = 1000, x.shape[1] // 2 - 7
    y = torch.zeros((1, 2, k1 - k0), dtype=torch.complex64, device="cuda")
    r.fir(TP._dev(x[None]), TP._dev(hw[None]), k0, k1, y)
    ref = chain.fir(x.astype(np.complex128), hw.astype(np.complex128), k0, k1)
    g = y[0].cpu().numpy()
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(g - ref)) < 1e-5 * rms


@pytest.mark.parametrize("case", ["qpsk80km", "gs1000km"])
def test_wl_cma_parity(case):
    st, p, res = TP._oracle_run(case)
    r = TP._receiver(case, widely_linear=1)
    x = res.x.astype(np.complex64)
    fmt = oracle_format(TP.CASES[case][0])
    h0 = chain.center_spike(p.taps, True)
    ref = chain.lms(x.astype(np.complex128), h0, range(2048), fmt, p, force_cma=True)
    taps = TP._dev(h0.astype(np.complex64)[None])
    r.lms(TP._dev(x[None]), taps, 0, 2048, None, 0, passes=1)
    g = taps[0].cpu().numpy()
    assert np.max(np.abs(g - ref)) < 2e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("P", [1, 16])
@pytest.mark.parametrize("case", ["qpsk80km", "gs1000km"])
def test_wl_dd_parity(case, P):
    st, p, res = TP._oracle_run(case)
    fmt = oracle_format(TP.CASES[case][0])
    x = res.x.astype(np.complex64)
    n = 2
    k0 = n * p.block
    h_in = _wl(res.taps_after[n - 1], np.random.default_rng(4), 0.01).astype(np.complex64)
    phase = {k: res.phi[k] for k in range(k0, k0 + p.n_upd)}
    p2 = chain.RxParams(**{**p.__dict__, "n_cma": 0})
    info = chain.LmsInfo()
    h128 = h_in.astype(np.complex128)
    span = range(k0, k0 + p.n_upd)
    if P == 1:
        ref = chain.lms(x.astype(np.complex128), h128, span, fmt, p2, phase=phase, info=info)
    else:
        ref = chain.lms_block(x.astype(np.complex128), h128, span, fmt, p2, P, phase=phase, info=info)
    if min(mg for _, mg in info.dd_margin) <= 1e-4:
        pytest.skip("oracle has a near-tie decision in the span")
    pcode = (res.b.astype(np.int64) | ((res.m % fmt.sym_order) << 8)).astype(np.uint16)
    r = TP._receiver(case, widely_linear=1, lms_block=P)
    taps = TP._dev(h_in[None])
    r.lms(TP._dev(x[None]), taps, k0, p.n_upd, TP._dev(pcode[None]), 1)
    g = taps[0].cpu().numpy()
    assert np.max(np.abs(g - ref)) < 2e-4 * np.max(np.abs(ref))


def _stream(seed, iq):
    fmt, n, cd, nfft, nov, T, B, blk, esn0, lw = CASE
    return synth.make_stream(fmt, n, seed=synth.stream_seed(13, seed), esn0_db=esn0, cd_ps_per_nm=cd,
                             linewidth_ts=lw, iq_imbalance=iq)


def _params(wl):
    fmt, n, cd, nfft, nov, T, B, blk, esn0, lw = CASE
    return chain.RxParams(cd_ps_per_nm=cd, n_fft=nfft, n_ov=nov, taps=T, bps_phases=B, block=blk, n_pre=4096,
                          widely_linear=wl)


def _receiver(wl):
    from paper_2108_07004_gb300 import rx
    fmt, n, cd, nfft, nov, T, B, blk, esn0, lw = CASE
    r = rx.Receiver(fmt, cd_ps_per_nm=cd, taps=T, bps_phases=B)
    for k, v in (("fft", nfft), ("overlap", nov), ("block", blk), ("n_pre", 4096), ("widely_linear", int(wl))):
        r.set(k, v)
    return r


def test_wl_chain_end_to_end():
    """The chain with the widely-linear butterfly against the oracle's, on a
    DP-16QAM stream with a transmitter IQ imbalance (segment protocol of the
    exact chain; the state carries 2T taps per branch)."""
    from paper_2108_07004_gb300 import rx
    st = _stream(1, IQ)
    p = _params(True)
    fmt = oracle_format(CASE[0])
    res = chain.run_chain(st.rx, fmt, p, ref_bits=st.bits)
    r = _receiver(True)
    r.set_reference(TP._dev(st.bits[None]))
    samples = TP._dev(st.rx[None])
    N = res.llr.shape[0]
    llr = torch.zeros((1, N, fmt.m), dtype=torch.float32, device="cuda")
    segs = TP._segments(res, p, N)
    for n0, n1 in segs:
        if n0 > 0:
            counters = rx.unpack_state(r.get_state())["counters"]
            stt = chain.state_at(res, p, n0)
            hd = dict(streams=1, taps=2 * p.taps, lag=p.lag, bps_window=p.bps_window, bps_phases=p.bps_phases,
                      m_bits=fmt.m, block=p.block, n_sym=N, blocks_done=n0, lms_updates=stt["lms_updates"])
            taps = np.stack([t[None] for t in stt["taps"]])
            r.set_state(rx.pack_state(hd, taps, np.array([stt["carry"]]), stt["y_tail"][None], counters))
        r.process_blocks(samples, n0, n1, llr)
    g = llr[0].cpu().numpy().astype(np.float64)
    fails = []
    for nb, (a, e) in enumerate(res.ranges):
        L0, dL, t_range, env = TP._block_valid(res, p, fmt, nb, N)
        fails += TP._check_block(g[a:e], L0, dL, t_range, env, a)
    assert not fails, f"segments {segs}: {len(fails)} rows fail: {fails[:4]}"


def test_wl_removes_the_iq_imbalance_penalty():
    """On the imbalanced stream without carrier phase noise (the regime of
    the paper's widely-linear equaliser: a KK receiver has none; 2^15
    symbols, blocks of 2048, the first 8192 symbols not counted) the
    widely-linear chain's bit errors are far below the linear chain's and
    near the linear chain's on the same stream without imbalance (the oracle
    gives 226 / 24 / 35).  With laser phase noise the conjugate term turns
    against the carrier before the phase search, so a butterfly in front of
    it cannot hold its conjugate taps."""
    from paper_2108_07004_gb300 import rx
    fmt, n, cd, nfft, nov, T, B, blk, esn0, lw = CASE
    out = {}
    for name, iq, wl in (("lin", IQ, False), ("wl", IQ, True), ("clean", None, False)):
        st = synth.make_stream(fmt, 1 << 15, seed=synth.stream_seed(13, 2), esn0_db=esn0, cd_ps_per_nm=cd,
                               linewidth_ts=0.0, iq_imbalance=iq)
        r = rx.Receiver(fmt, cd_ps_per_nm=cd, taps=T, bps_phases=B)
        for k, v in (("fft", nfft), ("overlap", nov), ("block", 2048), ("n_pre", 4096), ("skip_head", 8192),
                     ("widely_linear", int(wl))):
            r.set(k, v)
        r.set_reference(TP._dev(st.bits[None]))
        _, stats = r.process(TP._dev(st.rx[None]))
        out[name] = stats[0]["bit_errors"]
    assert out["wl"] * 3 < out["lin"], out
    assert out["wl"] < 1.6 * out["clean"] + 10, out
