"""The precision variant: the chain's CDC and FIR outputs stored as half or
bfloat16 pairs (float32 arithmetic, LMS and unwrap in float32), against the
FP64 oracle, stage by stage: EVM of the stored CDC output x and of the
stored FIR output y, error of the de-rotated symbols (EVM against the
oracle's z), the largest LLR error, and the BER against the oracle's.

Bounds follow the storage rounding: a stored sample carries a relative
error up to 2^-11 (half) or 2^-8 (bfloat16); x passes through the 31-tap
FIR and y is read again, so z carries about sqrt(2 * 31) rounding errors of
x-size plus one of y-size: relative RMS below 3 * 2^-11 (half) and 3 * 2^-8
(bfloat16) of |z| beside the float32 chain's own ~1e-6.  The stored x
itself carries one rounding (RMS below the unit of its format), and y the
FIR of x's roundings plus its own (below 3 units, as z)."""
import numpy as np
import pytest

from oracle import chain, oracle_format
from paper_2108_07004_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 1 << 14


@pytest.fixture(scope="module")
def case():
    st = synth.make_stream("gs4d64", N, seed=synth.stream_seed(3, 2), esn0_db=12.0,
                           cd_ps_per_nm=17000.0, linewidth_ts=2e-5)
    p = chain.RxParams(cd_ps_per_nm=17000.0, n_fft=4096, n_ov=1024, taps=31, bps_phases=64,
                       block=4096, n_pre=4096)
    res = chain.run_chain(st.rx, oracle_format("gs4d64"), p, ref_bits=st.bits)
    return st, p, res


def _run(st, prec):
    from paper_2108_07004_gb300 import rx
    r = rx.Receiver("gs4d64", cd_ps_per_nm=17000.0, taps=31, bps_phases=64)
    for k, v in (("fft", 4096), ("overlap", 1024), ("block", 4096), ("n_pre", 4096), ("precision", prec)):
        r.set(k, v)
    r.set_reference(torch.from_numpy(st.bits[None]).cuda())
    x4 = torch.zeros((1, N, 4), dtype=torch.float32, device="cuda")
    r.set_symbol_output(x4, None)
    llr, stats = r.process(torch.from_numpy(st.rx[None].astype(np.complex64)).cuda())
    z = x4[0].cpu().numpy().astype(np.float64)
    return llr[0].cpu().numpy().astype(np.float64), np.stack([z[:, 0] + 1j * z[:, 1], z[:, 2] + 1j * z[:, 3]]), stats[0]


@pytest.mark.parametrize("prec,unit", [(1, 2.0 ** -11), (2, 2.0 ** -8)])
def test_reduced_precision_storage_against_the_oracle(case, prec, unit):
    st, p, res = case
    llr, z, stats = _run(st, prec)
    llr32, z32, stats32 = _run(st, 0)
    same = res.bps_gap >= 1e-3                       # phase choices away from near-ties
    rows = np.arange(N) < res.ranges[1][1]           # taps shared with the oracle (blocks 0, 1)
    sel = same & rows
    ref = res.z[:, sel]
    evm = np.sqrt(np.mean(np.abs(z[:, sel] - ref) ** 2) / np.mean(np.abs(ref) ** 2))
    evm32 = np.sqrt(np.mean(np.abs(z32[:, sel] - ref) ** 2) / np.mean(np.abs(ref) ** 2))
    assert evm32 < 1e-5
    assert evm < 3 * unit, (evm, unit)
    err = np.abs(llr[sel] - res.llr[sel]) / np.maximum(1.0, np.abs(res.llr[sel]))
    assert np.max(err) < 100 * unit                  # sigma^2 and z both carry the storage error
    # bit errors within the binomial spread of the oracle's (~1000 errors at 12 dB)
    be, bo = stats["bit_errors"], res.stats["bit_errors"]
    assert abs(be - bo) <= 3 * np.sqrt(bo) + 3, (be, bo)


def test_state_needs_float32_storage(case):
    from paper_2108_07004_gb300 import rx
    st, _, _ = case
    r = rx.Receiver("gs4d64", cd_ps_per_nm=17000.0, taps=31, bps_phases=64)
    r.set("precision", 1)
    r.set("block", 4096)
    r.process_blocks(torch.from_numpy(st.rx[None].astype(np.complex64)).cuda(), 0, 1)
    with pytest.raises(rx.RxError) as e:
        r.get_state()
    assert e.value.code == -1


def _evm(a, ref):
    return float(np.sqrt(np.mean(np.abs(a - ref) ** 2) / np.mean(np.abs(ref) ** 2)))


def _pairs(t, prec):
    """[S][2][n] half / bfloat16 pairs (stored as int32 words) -> complex128."""
    dt = torch.float16 if prec == 1 else torch.bfloat16
    v = t.view(dt).float().cpu().numpy().astype(np.float64)
    return v[..., 0::2] + 1j * v[..., 1::2]


@pytest.mark.parametrize("prec,unit", [(1, 2.0 ** -11), (2, 2.0 ** -8)])
def test_stage_storage_error_cdc_and_fir(case, prec, unit):
    """Per stage: rx_cdc and rx_fir with the reduced storage (x stored, the
    FIR reading the stored x and storing y) against the oracle's x and its
    FIR with the same taps."""
    from paper_2108_07004_gb300 import rx
    st, p, res = case
    r = rx.Receiver("gs4d64", cd_ps_per_nm=17000.0, taps=31, bps_phases=64)
    for k, v in (("fft", 4096), ("overlap", 1024), ("precision", prec)):
        r.set(k, v)
    ns = st.rx.shape[1]
    x_in = torch.from_numpy(st.rx[None].astype(np.complex64)).cuda()
    xs = torch.zeros((1, 2, ns), dtype=torch.int32, device="cuda")       # 4-byte pairs
    r.cdc(x_in, xs)
    x = _pairs(xs, prec)[0]
    assert _evm(x, res.x) < unit, (_evm(x, res.x), unit)
    taps = res.taps_used[2]
    k0, k1 = 2 * p.block, 3 * p.block
    ys = torch.zeros((1, 2, k1 - k0), dtype=torch.int32, device="cuda")
    r.fir(xs, torch.from_numpy(taps.astype(np.complex64)[None]).cuda(), k0, k1, ys)
    y = _pairs(ys, prec)[0]
    ref = chain.fir(res.x, taps.astype(np.complex64).astype(np.complex128), k0, k1)
    assert _evm(y, ref) < 3 * unit, (_evm(y, ref), unit)
