"""Kramers-Kronig front-end on the GPU (rx_kk_field) against the FP64
oracle on the same ADC codes: several frames with a ragged tail, an odd
stream count (one stream without a partner in the two-streams-per-FFT
packing), both overlaps, a single short frame, and the full-size workload
on sampled streams.

Tolerance: the field is sqrt(I) e^{j phi} - A; in float32 the phase of a
1024-point FFT pair over ln|E| carries about 10 rounding steps of the
largest |ln|E|| (|ln I| / 2 < 3 here), i.e. ~2e-6 rad, and A = exp(mean
ln|E|) ~1e-7 relative, so |field_gpu - field_oracle| <= 2e-5 (A + |s|)
holds with margin."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mods():
    from paper_2108_07004_gb300 import rx, synth
    from oracle import kk as okk
    return rx, synth, okk


def _streams(synth, S, n_sym, seed0, cspr=12.0, esn0=20.0, fmt="dp_16qam"):
    ks = [synth.make_kk_stream(fmt, n_sym, seed=synth.stream_seed(60 + seed0, s), cspr_db=cspr,
                               esn0_db=esn0) for s in range(S)]
    codes = np.stack([k.codes for k in ks])
    levels = np.array([[k.scale, k.dc] for k in ks], dtype=np.float32)
    return ks, codes, levels


def _check(okk, ks, codes, levels, out, n_ov, floor, rows=None):
    rows = range(len(ks)) if rows is None else rows
    for s in rows:
        ref = okk.kk_field_from_codes(codes[s], scale=float(levels[s, 0]), dc=float(levels[s, 1]),
                                      fc_step=ks[s].fc_step, n_ov=n_ov, floor=floor)
        err = np.abs(out[s] - ref)
        bound = 2e-5 * (ks[s].carrier + np.abs(ref))
        assert np.all(err <= bound), (s, float(np.max(err / bound)))


@pytest.mark.parametrize("n_ov", [512, 256])
def test_kk_field_matches_oracle(n_ov):
    rx, synth, okk = _mods()
    S = 3
    ks, codes, levels = _streams(synth, S, 1400, 0)        # 5600 samples: 11 / 8 frames, ragged
    floor = float(np.float32(1e-3))
    k = rx.KK(ks[0].fc_step, n_ov=n_ov, floor=floor)
    out = k.field(torch.from_numpy(codes).cuda(), levels).cpu().numpy()
    _check(okk, ks, codes, levels, out, n_ov, floor)


def test_kk_short_stream_and_limits():
    rx, synth, okk = _mods()
    ks, codes, levels = _streams(synth, 1, 25, 1)           # 100 samples: one frame, mostly padding
    floor = float(np.float32(1e-3))
    k = rx.KK(ks[0].fc_step, n_ov=512, floor=floor)
    out = k.field(torch.from_numpy(codes).cuda(), levels).cpu().numpy()
    _check(okk, ks, codes, levels, out, 512, floor)
    # 256 streams in one call (the largest), checked on the first and last
    c = np.tile(codes, (256, 1))
    lv = np.tile(levels, (256, 1))
    out = k.field(torch.from_numpy(c).cuda(), lv).cpu().numpy()
    # the same pair of codes gives the same field in the same slot of a
    # stream pair (real or imaginary part of the packed FFT)
    assert np.array_equal(out[0], out[254]) and np.array_equal(out[1], out[255])
    _check(okk, [ks[0]] * 256, c, lv, out, 512, floor, rows=[0, 255])
    with pytest.raises(rx.RxError):
        k.field(torch.zeros((257, 8), dtype=torch.int16, device="cuda"), np.ones((257, 2)))
    with pytest.raises(rx.RxError):
        rx.KK(0, n_ov=1024)


def test_kk_full_size_sampled():
    """The benchmark's launch shape (32 streams of 2^22 samples), two
    streams checked whole against the oracle."""
    rx, synth, okk = _mods()
    S, n = 32, 1 << 22
    ks, codes, levels = _streams(synth, 2, n // 4, 2)
    c = np.concatenate([codes, np.tile(codes[1:], (S - 2, 1))])
    lv = np.concatenate([levels, np.tile(levels[1:], (S - 2, 1))])
    floor = float(np.float32(1e-3))
    k = rx.KK(ks[0].fc_step, n_ov=512, floor=floor)
    out_d = k.field(torch.from_numpy(c).cuda(), lv)
    out = out_d[[0, 1, S - 1]].cpu().numpy()
    # (a stream's rounding depends on its partner in the packed FFT, so the
    # last stream is checked against the oracle too, not for equality)
    _check(okk, [ks[0], ks[1], ks[1]], codes[[0, 1, 1]], levels[[0, 1, 1]], out, 512, floor)
