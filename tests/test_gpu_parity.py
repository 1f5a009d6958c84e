"""GPU parity: each stage of the CUDA library against the FP64 oracle.

Every test feeds the GPU the oracle's own inputs (cast to complex64) and
compares element by element.  Tolerances follow the FP32 arithmetic:
* CDC / FIR / de-rotation: complex64 sums of O(100) terms, relative RMS
  error ~1e-6; the bounds below leave 10-30x headroom.
* LLRs: |dLLR| <= 1e-4 * max(1, |LLR|) (the target tolerance of the chain).
* Integer results (phase indices, unwrap counts, bit errors): exact, except
  where the oracle itself has a near-tie, where either choice is valid and
  the choice must be within the tie.  BPS near-tie: relative gap between the
  two smallest window costs < 1e-4 (the FP32 window cost uses
  |y|^2 + |r|^2 - 2 max(|P|,|Q|) per symbol; at sigma^2 ~ 0.017 its relative
  error reaches ~1e-5).
* End to end: a near-tie inside a block's LMS span may send the taps of the
  following blocks along a different, equally valid trajectory; from the
  first block those taps reach, the GPU resumes from the oracle's block state
  (taps, unwrap carry, phase-search halo) and runs on from the samples.
"""
import numpy as np
import pytest

from oracle import chain, oracle_format
from paper_2108_07004_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from parity_protocol import DD_TIE, LLR_RTOL, TIE  # noqa: E402
from parity_protocol import block_valid as _block_valid  # noqa: E402
from parity_protocol import check_block as _check_block  # noqa: E402
from parity_protocol import segments as _segments  # noqa: E402


def _rx():
    from paper_2108_07004_gb300 import rx
    return rx


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


CASES = {
    # name: (format, n_sym, cd, n_fft, n_ov, taps, B, block, esn0, lw)
    "qpsk80km": ("dp_qpsk", 1 << 14, 1360.0, 1024, 256, 15, 32, 4096, 12.0, 1e-5),
    "gs1000km": ("gs4d64", 1 << 14, 17000.0, 4096, 1024, 31, 64, 4096, 12.0, 2e-5),
    "qam16": ("dp_16qam", 12000, 2000.0, 1024, 256, 15, 32, 4096, 18.0, 1e-5),
    "qam64": ("dp_64qam", 12000, 1000.0, 1024, 256, 15, 64, 4096, 24.0, 1e-6),
    "gs8": ("gs8", 12000, 500.0, 1024, 256, 15, 32, 4096, 14.0, 1e-5),
    # the paper's 128-point 2D GS format (Sec. 5): 32 orbits per polarisation
    # under the quarter-turn symmetry; at 30 dB the oracle's DD span has no
    # near-tie decision (the DD stage test needs none), and at the format's
    # 20 dB design point (BER ~4e-2) every test but the DD stage test runs
    "gs128": ("gs128", 12000, 500.0, 1024, 256, 15, 64, 4096, 30.0, 1e-6),
    "gs128_20db": ("gs128", 12000, 500.0, 1024, 256, 15, 64, 4096, 20.0, 1e-6),
    # the paper's receiver order: two single-polarisation KK signals (CSPR
    # 14 dB) through the KK front-end and the trained static equaliser
    # (oracle), then the chain as X and Y with the CDC reduced to the
    # identity (no dispersion, matched filtering done by the equaliser)
    "kk16": ("dp_16qam", 12000, 0.0, 1024, 256, 15, 32, 4096, 20.0, 0.0),
}
KK_CASES = {"kk16"}
DD_NEAR_TIE_CASES = {"gs128_20db"}


def _kk_input(n_sym, seed, esn0):
    """[2, 2N] complex64 samples and [N, 8] bits: KK field and trained
    static equaliser (oracle) of two independent 16QAM KK streams."""
    from types import SimpleNamespace
    from oracle import fde, kk
    ys, bits = [], []
    for q in range(2):
        k = synth.make_kk_stream("dp_16qam", n_sym, seed=seed + q, cspr_db=14.0, esn0_db=esn0)
        x = kk.kk_field_from_codes(k.codes, scale=k.scale, dc=k.dc, fc_step=k.fc_step, floor=1e-3)
        h = fde.train(x, k.sym[:4096])
        ys.append(fde.apply(x, h))
        bits.append(k.bits)
    return SimpleNamespace(rx=np.stack(ys).astype(np.complex64), bits=np.concatenate(bits, axis=1))


def _params(case):
    fmt, n, cd, nfft, nov, T, B, blk, esn0, lw = CASES[case]
    return chain.RxParams(cd_ps_per_nm=cd, n_fft=nfft, n_ov=nov, taps=T, bps_phases=B,
                          block=blk, n_pre=4096, matched_filter=case not in KK_CASES)


_cache = {}


def _oracle_run(case):
    if case not in _cache:
        fmt, n, cd, nfft, nov, T, B, blk, esn0, lw = CASES[case]
        if case in KK_CASES:
            st = _kk_input(n, synth.stream_seed(9, 50), esn0)
        else:
            st = synth.make_stream(fmt, n, seed=synth.stream_seed(9, len(_cache)), esn0_db=esn0,
                                   cd_ps_per_nm=cd, linewidth_ts=lw)
        p = _params(case)
        res = chain.run_chain(st.rx, oracle_format(fmt), p, ref_bits=st.bits)
        _cache[case] = (st, p, res)
    return _cache[case]


def _receiver(case, **kw):
    rx = _rx()
    fmt, n, cd, nfft, nov, T, B, blk, esn0, lw = CASES[case]
    r = rx.Receiver(fmt, cd_ps_per_nm=cd, taps=T, bps_phases=B)
    r.set("fft", nfft)
    r.set("overlap", nov)
    r.set("block", blk)
    r.set("n_pre", 4096)
    if case in KK_CASES:
        r.set("matched_filter", 0)
    for k, v in kw.items():
        r.set(k, v)
    return r


@pytest.mark.parametrize("case", list(CASES))
def test_cdc_parity(case):
    st, p, res = _oracle_run(case)
    r = _receiver(case)
    x_in = _dev(st.rx[None])
    out = torch.zeros_like(x_in)
    r.cdc(x_in, out)
    torch.cuda.synchronize()
    g = out[0].cpu().numpy().astype(np.complex128)
    ref = res.x
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    err = np.abs(g - ref)
    assert np.sqrt(np.mean(err ** 2)) < 3e-6 * rms
    assert err.max() < 3e-5 * rms


def test_cdc_ragged_and_multistream():
    """Several streams at once; a length that ends inside a frame."""
    rx = _rx()
    p = chain.RxParams(cd_ps_per_nm=500.0, n_fft=1024, n_ov=256)
    S, ns = 3, 5000 * 2 + 2          # ragged: not a multiple of the 768-sample hop
    rng = np.random.default_rng(1)
    xs = (rng.standard_normal((S, 2, ns)) + 1j * rng.standard_normal((S, 2, ns))).astype(np.complex64)
    r = rx.Receiver("dp_qpsk", cd_ps_per_nm=500.0, taps=15, bps_phases=32, streams=S)
    out = torch.zeros((S, 2, ns), dtype=torch.complex64, device="cuda")
    r.cdc(_dev(xs), out)
    g = out.cpu().numpy()
    for s in range(S):
        ref = chain.cdc(xs[s].astype(np.complex128), p)
        assert np.max(np.abs(g[s] - ref)) < 3e-5 * np.sqrt(np.mean(np.abs(ref) ** 2))


@pytest.mark.parametrize("case", list(CASES))
def test_fir_parity(case):
    st, p, res = _oracle_run(case)
    r = _receiver(case)
    x = res.x.astype(np.complex64)
    rng = np.random.default_rng(2)
    T = p.taps
    taps = (res.w0 + 0.05 * (rng.standard_normal((2, 2, T)) + 1j * rng.standard_normal((2, 2, T))))
    k0, k1 = 1000, x.shape[1] // 2 - 7      # ragged end, interior start
    y = torch.zeros((1, 2, k1 - k0), dtype=torch.complex64, device="cuda")
    r.fir(_dev(x[None]), _dev(taps.astype(np.complex64)[None]), k0, k1, y)
    ref = chain.fir(x.astype(np.complex128), taps.astype(np.complex64).astype(np.complex128), k0, k1)
    g = y[0].cpu().numpy()
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(g - ref)) < 1e-5 * rms


@pytest.mark.parametrize("case", list(CASES))
def test_lms_cma_parity(case):
    """Start-up CMA (two passes) from the identity on the oracle's CDC output."""
    st, p, res = _oracle_run(case)
    r = _receiver(case)
    x = res.x.astype(np.complex64)
    fmt = oracle_format(CASES[case][0])
    h0 = chain.center_spike(p.taps)
    ref = h0
    for _ in range(2):
        ref = chain.lms(x.astype(np.complex128), ref, range(2048), fmt, p, force_cma=True)
    taps = _dev(h0.astype(np.complex64)[None])
    r.lms(_dev(x[None]), taps, 0, 2048, None, 0, passes=2)
    g = taps[0].cpu().numpy()
    assert np.max(np.abs(g - ref)) < 2e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("case", list(CASES))
def test_lms_dd_parity(case):
    """DD-LMS of one block span with the oracle's taps and phases."""
    if case in DD_NEAR_TIE_CASES:
        pytest.skip("the oracle's DD span holds near-tie decisions at this operating point")
    st, p, res = _oracle_run(case)
    r = _receiver(case)
    fmt = oracle_format(CASES[case][0])
    x = res.x.astype(np.complex64)
    n = 2          # block index with DD updates (n_cma = 1024 -> block 0 span is CMA)
    k0 = n * p.block
    h_in = res.taps_after[n - 1].astype(np.complex64)
    phase = {k: res.phi[k] for k in range(k0, k0 + p.n_upd)}
    p2 = chain.RxParams(**{**p.__dict__, "n_cma": 0})
    info = chain.LmsInfo()
    ref = chain.lms(x.astype(np.complex128), h_in.astype(np.complex128), range(k0, k0 + p.n_upd),
                    fmt, p2, phase=phase, info=info)
    assert min(mg for _, mg in info.dd_margin) > 1e-4, "oracle has a near-tie decision"
    pcode = (res.b.astype(np.int64) | ((res.m % fmt.sym_order) << 8)).astype(np.uint16)
    taps = _dev(h_in[None])
    r.lms(_dev(x[None]), taps, k0, p.n_upd, _dev(pcode[None]), 1)
    g = taps[0].cpu().numpy()
    assert np.max(np.abs(g - ref)) < 2e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("case", list(CASES))
def test_training_stage_parity(case):
    """Order/phase alignment, data-aided phase codes and data-aided LMS from
    the oracle's start-up CMA taps."""
    st, p, res = _oracle_run(case)
    r = _receiver(case)
    fmt = oracle_format(CASES[case][0])
    r.set_reference(_dev(st.bits[None]))
    x = res.x.astype(np.complex64)
    taps = _dev(res.w_cma.astype(np.complex64)[None])
    ntr = p.n_train
    pc = torch.zeros((1, ntr), dtype=torch.int16, device="cuda")
    r.train(_dev(x[None]), taps, pc)
    torch.cuda.synchronize()
    code = pc[0].cpu().numpy().astype(np.int64) & 0xFFFF
    S = fmt.sym_order
    same = (code & 255) == res.train_b
    same &= (code >> 8) == (res.train_m % S)
    assert same.mean() > 0.995          # codes that differ sit on a rounding boundary
    g = taps[0].cpu().numpy()
    assert np.max(np.abs(g - res.w0)) < 1e-3 * np.max(np.abs(res.w0))


@pytest.mark.parametrize("case", list(CASES))
def test_bps_parity(case):
    st, p, res = _oracle_run(case)
    r = _receiver(case)
    fmt = oracle_format(CASES[case][0])
    y = res.y.astype(np.complex64)
    N = y.shape[1]
    a, e = 37, N - 101            # ragged range, windows truncated at n_valid = N
    b_ref, gap, _ = chain.bps(y.astype(np.complex128), a, e, N, p, fmt)
    bo = torch.zeros((1, e - a), dtype=torch.uint8, device="cuda")
    r.bps(_dev(y[None]), a, e, N, bo)
    g = bo[0].cpu().numpy().astype(np.int64)
    diff = g != b_ref
    assert np.all(gap[diff] < TIE), f"{diff.sum()} choices differ outside near-ties"
    assert diff.mean() < 1e-3


@pytest.mark.parametrize("case", list(CASES))
def test_unwrap_parity(case):
    st, p, res = _oracle_run(case)
    r = _receiver(case)
    fmt = oracle_format(CASES[case][0])
    N = res.y.shape[1]
    y = res.y.astype(np.complex64)
    a, e = res.ranges[1]
    b = res.b[a:e].astype(np.uint8)
    # carry from the oracle's previous range
    a0, e0 = res.ranges[0]
    carry = np.array([[res.m[e0 - 1], res.b[e0 - 1]]], dtype=np.int32)
    z = torch.zeros((1, 2, e - a), dtype=torch.complex64, device="cuda")
    pc = torch.zeros((1, e - a), dtype=torch.int16, device="cuda")
    cout = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    s2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    r.unwrap(_dev(y[None]), _dev(b[None]), a, e, _dev(carry), z, pc, cout, s2)
    torch.cuda.synchronize()
    S = fmt.sym_order
    code = pc[0].cpu().numpy().astype(np.int64) & 0xFFFF
    assert np.array_equal(code & 255, res.b[a:e])
    assert np.array_equal(code >> 8, res.m[a:e] % S)
    assert cout[0, 0].item() % S == res.m[e - 1] % S and cout[0, 1].item() == res.b[e - 1]
    gz = z[0].cpu().numpy()
    assert np.max(np.abs(gz - res.z[:, a:e])) < 1e-5 * np.max(np.abs(res.z[:, a:e]))
    assert abs(s2.item() / res.sigma2[1] - 1) < 1e-5


@pytest.mark.parametrize("case", list(CASES))
def test_demap_parity(case):
    st, p, res = _oracle_run(case)
    r = _receiver(case)
    fmt = oracle_format(CASES[case][0])
    z = res.z.astype(np.complex64)
    K = z.shape[1]
    s2 = 0.07
    llr = torch.zeros((1, K, fmt.m), dtype=torch.float32, device="cuda")
    r.demap(_dev(z[None]), torch.tensor([s2], dtype=torch.float64, device="cuda"), llr)
    ref = chain.llr(z.astype(np.complex128), s2, fmt)
    g = llr[0].cpu().numpy().astype(np.float64)
    err = np.abs(g - ref)
    assert np.all(err <= LLR_RTOL * np.maximum(1.0, np.abs(ref)))


@pytest.mark.parametrize("name", ["gs4d64", "dp_16qam", "dp_qpsk", "dp_64qam", "gs8", "gs128"])
def test_demap_extreme_llrs(name):
    """Subset sums beyond the float range of the common shift use their own
    shift: every symbol extreme (small sigma^2), and a ragged length with
    every 7th symbol at twice its amplitude, so that every warp mixes
    extreme and ordinary lanes (and the last warp has lanes past the end)."""
    rx = _rx()
    fmt = oracle_format(name)
    rng = np.random.default_rng(5)
    n = 509
    bits = rng.integers(0, 2, size=(n, fmt.m), dtype=np.uint8)
    z = fmt.symbols_from_bits(bits) + 0.02 * (rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n)))
    zf = z.copy()
    zf[:, ::7] *= 2.0
    kw = dict(taps=31, bps_phases=64) if fmt.dims == 4 else dict(taps=15, bps_phases=32)
    r = rx.Receiver(name, **kw)
    for zz, s2 in ((z, 1e-3), (z, 3e-3), (zf, 0.02)):
        zz = zz.astype(np.complex64)
        llr = torch.zeros((1, n, fmt.m), dtype=torch.float32, device="cuda")
        r.demap(_dev(zz[None]), torch.tensor([s2], dtype=torch.float64, device="cuda"), llr)
        ref = chain.llr(zz.astype(np.complex128), s2, fmt)
        g = llr[0].cpu().numpy().astype(np.float64)
        assert np.abs(ref).max() > 200          # past the common shift's range
        bad = np.abs(g - ref) > LLR_RTOL * np.maximum(1.0, np.abs(ref))
        assert not bad.any(), (s2, np.flatnonzero(bad.any(axis=1))[:10])


def _oracle_state(rx, res, p, fmt, n, N, counters):
    stt = chain.state_at(res, p, n)
    hd = dict(streams=1, taps=p.taps, lag=p.lag, bps_window=p.bps_window, bps_phases=p.bps_phases,
              m_bits=fmt.m, block=p.block, n_sym=N, blocks_done=n, lms_updates=stt["lms_updates"])
    taps = np.stack([t[None] for t in stt["taps"]])
    return rx.pack_state(hd, taps, np.array([stt["carry"]]), stt["y_tail"][None], counters)


def test_bps_parity_tensor_cores():
    """The 4D-64 phase search with the orbit correlations on the tensor cores
    (bps_tc = 1) against the oracle: exact outside near-ties."""
    st, p, res = _oracle_run("gs1000km")
    r = _receiver("gs1000km", bps_tc=1)
    fmt = oracle_format("gs4d64")
    y = res.y.astype(np.complex64)
    N = y.shape[1]
    a, e = 37, N - 101
    b_ref, gap, _ = chain.bps(y.astype(np.complex128), a, e, N, p, fmt)
    bo = torch.zeros((1, e - a), dtype=torch.uint8, device="cuda")
    r.bps(_dev(y[None]), a, e, N, bo)
    g = bo[0].cpu().numpy().astype(np.int64)
    diff = g != b_ref
    assert np.all(gap[diff] < TIE), f"{diff.sum()} choices differ outside near-ties"
    assert diff.mean() < 1e-3


def test_chain_end_to_end_tensor_cores():
    """The 4D-64 chain with the tensor-core phase search, same protocol."""
    st, p, res = _oracle_run("gs1000km")
    _e2e_check("gs1000km", st, p, res, _receiver("gs1000km", bps_tc=1))


@pytest.mark.parametrize("case", list(CASES))
def test_chain_end_to_end(case):
    """rx_process_blocks against the oracle's block schedule on the same
    stream.  The GPU starts the stream itself (start-up CMA, training, block
    0, ...) and runs on from the samples; after a near-tie in an LMS span it
    resumes, lag blocks later, from the oracle's state (rx_set_state).  Every
    row is compared, against the envelope of the LLRs that the valid choices
    at BPS near-ties allow (exactly the oracle's LLR where a block has none)."""
    st, p, res = _oracle_run(case)
    _e2e_check(case, st, p, res, _receiver(case))


@pytest.mark.parametrize("case", ["qpsk80km", "qam16", "gs1000km"])
def test_chain_end_to_end_independent_lms_chains(case):
    """lms_start = 1 at lag 3: the update of block n starts from the taps
    that equalised it, and the three interleaved chains run concurrently on
    three streams; the same protocol against the oracle's schedule."""
    st, _, _ = _oracle_run(case)
    p = _params(case)
    p.lag, p.lms_start = 3, 1
    res = chain.run_chain(st.rx, oracle_format(CASES[case][0]), p, ref_bits=st.bits)
    _e2e_check(case, st, p, res, _receiver(case, lag=3, lms_start=1))


def _e2e_check(case, st, p, res, r):
    rx = _rx()
    fmt = oracle_format(CASES[case][0])
    r.set_reference(_dev(st.bits[None]))
    samples = _dev(st.rx[None])
    N = res.llr.shape[0]
    llr = torch.zeros((1, N, fmt.m), dtype=torch.float32, device="cuda")
    segs = _segments(res, p, N)
    for n0, n1 in segs:
        if n0 > 0:
            counters = rx.unpack_state(r.get_state())["counters"]    # the GPU's own counts go on
            r.set_state(_oracle_state(rx, res, p, fmt, n0, N, counters))
        _, stats = r.process_blocks(samples, n0, n1, llr)
    g = llr[0].cpu().numpy().astype(np.float64)
    ref = res.llr
    tie = res.bps_gap < TIE
    fails = []
    amb = np.abs(ref) < 1e-4
    for n, (a, e) in enumerate(res.ranges):
        L0, dL, t_range, env = _block_valid(res, p, fmt, n, N)
        fails += _check_block(g[a:e], L0, dL, t_range, env, a)
        t_max = max(abs(t_range[0]), abs(t_range[1]))
        amb[a:e] |= np.abs(L0) <= 1e-4 + np.abs(dL) * t_max
        for k, (lo, hi) in env.items():
            amb[k] |= (lo <= 1e-4) & (hi >= -1e-4)
    assert not fails, f"segments {segs}: {len(fails)} rows fail: {fails[:6]}"
    # hard decisions identical except where a valid LLR is within 1e-4 of 0
    hd = ((g < 0) != (ref < 0)) & ~amb
    assert hd.sum() == 0
    # counting: bit errors of the GPU's own hard decisions are exact
    c0, c1 = p.skip_head, N - p.skip_tail
    mine = int(np.sum((g[c0:c1] < 0).astype(np.uint8) != st.bits[c0:c1]))
    assert stats[0]["bit_errors"] == mine
    if not tie[c0:c1].any():
        assert stats[0]["bit_errors"] == res.stats["bit_errors"]
        assert abs(stats[0]["gmi"] - res.stats["gmi"]) < 1e-4 * fmt.m