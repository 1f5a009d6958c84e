"""Static frequency-domain equaliser on the GPU (rx_fde_*) against the FP64
oracle: float64 least-squares training, overlap-save application with
4 -> 2 resampling, and the paper's order KK front-end -> trained static
equaliser on the GPU end to end.

Tolerances.  Training runs in float64 on both sides from the same float32
inputs; only the summation order differs, amplified by the condition
number of R + lam I (at most T / delta = 2e8 for delta = 1e-6), so the taps
agree to 1e-6 relative.  Application is float32: two 1024-point FFTs
(about 20 rounding steps of 6e-8 on values of the frame's rms), so
|y_gpu - y_oracle| <= 2e-5 (rms(y) + |y|)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mods():
    from paper_2108_07004_gb300 import rx, synth
    from oracle import fde as ofde, kk as okk
    return rx, synth, ofde, okk


def _kk_field(synth, okk, n_sym, seed, cspr=14.0, esn0=25.0):
    k = synth.make_kk_stream("dp_16qam", n_sym, seed=seed, cspr_db=cspr, esn0_db=esn0)
    x = okk.kk_field_from_codes(k.codes, scale=k.scale, dc=k.dc, fc_step=k.fc_step, floor=1e-3)
    return k, x.astype(np.complex64)


def test_fde_training_matches_oracle():
    rx, synth, ofde, okk = _mods()
    k, x = _kk_field(synth, okk, 6000, synth.stream_seed(70, 0))
    d = k.sym[:4096].astype(np.complex64)
    e = rx.FDE(203, 256)
    e.train(torch.from_numpy(x).cuda(), torch.from_numpy(d).cuda(), sps=4, delta=1e-6)
    h = e.taps()
    h_ref = ofde.train(x.astype(np.complex128), d.astype(np.complex128), T=203, sps=4, delta=1e-6)
    assert np.linalg.norm(h - h_ref) <= 1e-6 * np.linalg.norm(h_ref)
    # a short equaliser and another oversampling
    e2 = rx.FDE(31, 256)
    e2.train(torch.from_numpy(x).cuda(), torch.from_numpy(d[:1000]).cuda(), sps=4, delta=1e-3)
    h2 = ofde.train(x.astype(np.complex128), d[:1000].astype(np.complex128), T=31, sps=4, delta=1e-3)
    assert np.linalg.norm(e2.taps() - h2) <= 1e-6 * np.linalg.norm(h2)


@pytest.mark.parametrize("n_ov", [256, 512])
def test_fde_apply_matches_oracle(n_ov):
    rx, synth, ofde, okk = _mods()
    S = 3
    xs = [_kk_field(synth, okk, 1700, synth.stream_seed(71, s))[1] for s in range(S)]   # 6800 samples, ragged
    x = np.stack(xs)
    rng = np.random.default_rng(5)
    h = (rng.standard_normal(203) + 1j * rng.standard_normal(203)) * np.exp(-np.abs(np.arange(203) - 101) / 20)
    e = rx.FDE(203, n_ov)
    e.set_taps(h)
    assert np.array_equal(e.taps(), h)
    y = e.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    for s in range(S):
        ref = ofde.apply(x[s].astype(np.complex128), h, n_ov=n_ov)
        rms = np.sqrt(np.mean(np.abs(ref) ** 2))
        assert np.all(np.abs(y[s] - ref) <= 2e-5 * (rms + np.abs(ref)))


def test_kk_then_fde_on_gpu():
    """KK front-end, training and application all on the GPU: outputs agree
    with the oracle chain and the symbol-instant EVM matches to 0.05 dB."""
    rx, synth, ofde, okk = _mods()
    k = synth.make_kk_stream("dp_16qam", 8192, seed=synth.stream_seed(72, 0), cspr_db=14.0, esn0_db=25.0)
    floor = float(np.float32(1e-3))
    kkh = rx.KK(k.fc_step, n_ov=512, floor=floor)
    xg = kkh.field(torch.from_numpy(k.codes[None]).cuda(), [[k.scale, k.dc]])
    e = rx.FDE(203, 256)
    d = torch.from_numpy(k.sym[:4096].astype(np.complex64)).cuda()
    e.train(xg[0], d)
    y = e.apply(xg)[0].cpu().numpy()
    x_o = okk.kk_field_from_codes(k.codes, scale=k.scale, dc=k.dc, fc_step=k.fc_step, floor=floor)
    h_o = ofde.train(x_o, k.sym[:4096])
    y_o = ofde.apply(x_o, h_o)
    rms = np.sqrt(np.mean(np.abs(y_o) ** 2))
    assert np.max(np.abs(y - y_o)) <= 1e-3 * rms
    sl = slice(100, -100)
    p = np.mean(np.abs(k.sym) ** 2)
    evm = 10 * np.log10(np.mean(np.abs(y[0::2][sl] - k.sym[sl]) ** 2) / p)
    evm_o = 10 * np.log10(np.mean(np.abs(y_o[0::2][sl] - k.sym[sl]) ** 2) / p)
    assert abs(evm - evm_o) < 0.05 and evm < -20.0


def test_fde_rejections():
    rx, *_ = _mods()
    with pytest.raises(rx.RxError):
        rx.FDE(204, 256)                      # even taps
    with pytest.raises(rx.RxError):
        rx.FDE(301, 256)                      # longer than the overlap
    e = rx.FDE(203, 256)
    x = torch.zeros((1, 1000), dtype=torch.complex64, device="cuda")
    with pytest.raises(rx.RxError):
        e.apply(x)                            # no taps yet
    e.set_taps(np.eye(1, 203, 101)[0])
    with pytest.raises(rx.RxError):
        e.apply(torch.zeros((1, 999), dtype=torch.complex64, device="cuda"))
