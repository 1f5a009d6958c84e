"""The paper's receiver order entirely on the GPU: two single-polarisation
KK signals -> KK front-end -> trained static equaliser (4 -> 2 samples per
symbol) -> the chain with the CDC reduced to the identity, against the same
pipeline in the oracle on the same ADC codes.

Each stage's elementwise parity is tested on its own (test_gpu_kk,
test_gpu_fde, and the chain on the oracle's equaliser output in
test_gpu_parity's kk16 case).  Here the inputs of each GPU stage carry the
previous GPU stages' float32 rounding (about 1e-6 relative), which can move
decisions at near-ties only, so the comparison is of the counts: bit errors
within max(3, 5 %) and GMI within 2e-3 bit per 4D symbol."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_kk_receiver_pipeline_matches_oracle():
    from paper_2108_07004_gb300 import rx, synth
    from oracle import chain, fde, kk, oracle_format
    n = 16384
    ks = [synth.make_kk_stream("dp_16qam", n, seed=synth.stream_seed(73, q), cspr_db=14.0, esn0_db=19.0)
          for q in range(2)]
    floor = float(np.float32(1e-3))
    bits = np.concatenate([ks[0].bits, ks[1].bits], axis=1)
    p = chain.RxParams(cd_ps_per_nm=0.0, n_fft=1024, n_ov=256, taps=15, bps_phases=32, block=4096,
                       n_pre=4096, matched_filter=False)
    ys = []
    for k in ks:
        x = kk.kk_field_from_codes(k.codes, scale=k.scale, dc=k.dc, fc_step=k.fc_step, floor=floor)
        ys.append(fde.apply(x, fde.train(x, k.sym[:4096])))
    res = chain.run_chain(np.stack(ys).astype(np.complex64), oracle_format("dp_16qam"), p, ref_bits=bits)

    kkh = rx.KK(ks[0].fc_step, n_ov=512, floor=floor)
    field = kkh.field(torch.from_numpy(np.stack([k.codes for k in ks])).cuda(),
                      [[k.scale, k.dc] for k in ks])
    y = torch.empty((2, 2 * n), dtype=torch.complex64, device="cuda")
    for q, k in enumerate(ks):
        e = rx.FDE(203, 256)
        e.train(field[q], torch.from_numpy(k.sym[:4096].astype(np.complex64)).cuda())
        e.apply(field[q:q + 1], y[q:q + 1])
    r = rx.Receiver("dp_16qam", cd_ps_per_nm=0.0, taps=15, bps_phases=32)
    for key, v in (("fft", 1024), ("overlap", 256), ("block", 4096), ("n_pre", 4096), ("matched_filter", 0)):
        r.set(key, v)
    r.set_reference(torch.from_numpy(bits[None]).cuda())
    _, st = r.process(y.view(1, 2, 2 * n))
    ne_g, ne_o = st[0]["bit_errors"], res.stats["bit_errors"]
    assert st[0]["n_bits"] == res.stats["n_bits"]
    assert ne_o > 0
    assert abs(ne_g - ne_o) <= max(3, 0.05 * ne_o), (ne_g, ne_o)
    assert abs(st[0]["gmi"] - res.stats["gmi"]) < 2e-3
