"""GPU parity of the learned demapper (MLP 4 -> 128 -> 128 -> 6) against the
FP64 oracle: gradients, one Adam step, inference, and a training run on the
GPU's own forward and backward kernels.

Tolerances: the GPU computes with the same bfloat16-rounded weights as the
oracle, float32 activations and float32 sums over the batch, so gradients
agree to float32 summation error (1e-4 of each parameter group's largest
entry) and LLRs to 1e-4 * max(1, |LLR|)."""
import math

import numpy as np
import pytest

from oracle import chain, mlp, oracle_format

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rx():
    from paper_2108_07004_gb300 import rx
    return rx


def _awgn(n, esn0, seed):
    fmt = oracle_format("gs4d64")
    r = np.random.default_rng(seed)
    bits = r.integers(0, 2, size=(n, 6), dtype=np.uint8)
    s = fmt.symbols_from_bits(bits)
    n0 = 10 ** (-esn0 / 10)
    z = s + math.sqrt(n0 / 2) * (r.standard_normal(s.shape) + 1j * r.standard_normal(s.shape))
    x = np.stack([z[0].real, z[0].imag, z[1].real, z[1].imag], axis=1)
    return x, np.full(n, n0), bits, z


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).cuda()


def _params(seed):
    th = mlp.init_params(seed)
    p = mlp.unpack(th)
    rng = np.random.default_rng(seed + 1)
    for b in ("b1", "b2", "b3"):
        p[b][:] = (rng.standard_normal(p[b].shape) * 0.1).astype(np.float32)
    return th


@pytest.mark.parametrize("train_tc", [1, 0])
@pytest.mark.parametrize("n", [777, 4096])
def test_gradient_matches_oracle(n, train_tc):
    """Both GEMM paths: tcgen05 with three-term bfloat16 operands (ragged
    batch 777: a partial 128-row tile and a partial 256-sample dW2 slice)
    and the float32 SIMT GEMMs."""
    rx = _rx()
    th = _params(3)
    x, s2, bits, _ = _awgn(n, 10.0, 4)
    m = rx.Mlp(th)
    m.set_param("train_tc", train_tc)
    assert m.get_param("train_tc") == train_tc
    g, loss = m.grad(_dev(x, np.float32), _dev(s2, np.float32), _dev(bits, np.uint8))
    torch.cuda.synchronize()
    w = mlp.compute_weights(th)
    ref_loss, ref = mlp.loss_and_grad(w, x.astype(np.float32).astype(np.float64),
                                      s2.astype(np.float32).astype(np.float64), bits)
    gg = mlp.unpack(g.cpu().numpy().astype(np.float64))
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    for name, _ in mlp.SHAPES:
        scale = np.max(np.abs(ref[name]))
        assert np.max(np.abs(gg[name] - ref[name])) <= 1e-4 * scale, name


def test_adam_step_matches_oracle():
    rx = _rx()
    th = _params(5)
    x, s2, bits, _ = _awgn(1024, 10.0, 6)
    m = rx.Mlp(th)
    m.train_step(_dev(x, np.float32), _dev(s2, np.float32), _dev(bits, np.uint8), 1e-3)
    got = m.params().astype(np.float64)
    w = mlp.compute_weights(th)
    _, g = mlp.loss_and_grad(w, x.astype(np.float32).astype(np.float64),
                             s2.astype(np.float32).astype(np.float64), bits)
    want = mlp.Adam(lr=1e-3).step(th.astype(np.float64), mlp.pack(g))
    step = np.abs(want - th)
    gmax = np.abs(mlp.pack(g))
    clear = gmax > 1e-3 * np.max(gmax)            # the first step is lr * sign(g) there
    assert np.max(np.abs(got - want)[clear]) <= 1e-6
    assert np.all(np.abs(got - th) <= 1e-3 * (1 + 1e-5) + 1e-7)   # no step exceeds lr
    assert np.all(step <= 1e-3 * (1 + 1e-6))


@pytest.mark.parametrize("path", [2, 1])
@pytest.mark.parametrize("n", [5000, 200_003])
def test_inference_matches_oracle(n, path):
    """tcgen05 (2) and mma.sync (1) inference; 5000 samples end in a partial
    128-sample tile, 200 003 give the persistent blocks several tiles each."""
    rx = _rx()
    th = _params(7)
    x, s2, bits, _ = _awgn(n, 12.0, 8)
    s2 = s2 * np.linspace(0.5, 2.0, s2.size)                  # per-symbol sigma^2
    m = rx.Mlp(th)
    m.set_param("infer", path)
    llr = m.infer(_dev(x, np.float32), _dev(s2, np.float32)).cpu().numpy().astype(np.float64)
    ref = mlp.llr(mlp.compute_weights(th), x.astype(np.float32).astype(np.float64),
                  s2.astype(np.float32).astype(np.float64))
    assert np.all(np.abs(llr - ref) <= 1e-4 * np.maximum(1.0, np.abs(ref)))


def test_training_on_the_gpu_gains_over_the_untrained_network():
    """Adam on the GPU's own forward and backward kernels (2^15 AWGN 4D-64
    symbols at 12 dB, batch 1024): the loss falls, the GMI rises from far
    below zero to within 0.3 bit of the exact log-sum-exp demapper, and the
    run is reproducible bit for bit."""
    rx = _rx()
    x, s2, bits, _ = _awgn(1 << 15, 12.0, 9)
    xt, s2t, bt, zt = _awgn(1 << 13, 12.0, 10)
    fmt = oracle_format("gs4d64")
    exact = chain.count(chain.llr(zt, s2t[0], fmt), bt.astype(float))["gmi"]
    X, S2, BT = _dev(x, np.float32), _dev(s2, np.float32), _dev(bits, np.uint8)
    Xt, S2t = _dev(xt, np.float32), _dev(s2t, np.float32)
    results = []
    for _ in range(2):
        m = rx.Mlp(mlp.init_params(11))
        before = chain.count(m.infer(Xt, S2t).cpu().numpy().astype(np.float64), bt.astype(float))["gmi"]
        rng = np.random.default_rng(0)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        losses = []
        for step in range(600):
            idx = torch.from_numpy(rng.integers(0, x.shape[0], size=1024)).cuda()
            m.train_step(X[idx].contiguous(), S2[idx].contiguous(), BT[idx].contiguous(), 3e-3, loss)
            if step % 100 == 0 or step == 599:
                losses.append(loss.item())
        after = chain.count(m.infer(Xt, S2t).cpu().numpy().astype(np.float64), bt.astype(float))["gmi"]
        results.append((m.params(), losses, before, after))
    (p0, l0, b0, a0), (p1, l1, _, _) = results
    assert np.array_equal(p0, p1) and l0 == l1                 # deterministic
    assert l0[-1] < l0[0] / 20
    assert b0 < 0.0 and exact - 0.3 < a0 < exact + 0.01


@pytest.mark.parametrize("S", [1, 3])
def test_chain_with_learned_demapper_and_symbol_output(S):
    """The chain's symbol output does not change its LLRs; with the learned
    demapper the chain's LLRs are the MLP's on those symbols (one inference
    launch per block over the S streams) and its bit counts are those of its
    own hard decisions."""
    rx = _rx()
    from paper_2108_07004_gb300 import synth
    n = 20000
    sts = [synth.make_stream("gs4d64", n, seed=synth.stream_seed(4, 1 + s), esn0_db=13.0 - s,
                             cd_ps_per_nm=17000.0, linewidth_ts=2e-5) for s in range(S)]
    samples = _dev(np.stack([st.rx for st in sts]), np.complex64)
    bits = _dev(np.stack([st.bits for st in sts]), np.uint8)

    def receiver():
        r = rx.Receiver("gs4d64", cd_ps_per_nm=17000.0, taps=31, bps_phases=64)
        for k, v in (("fft", 4096), ("overlap", 1024), ("block", 4096), ("n_pre", 4096), ("streams", S)):
            r.set(k, v)
        r.set_reference(bits)
        return r

    ref, st_ref = receiver().process(samples)
    r = receiver()
    x4 = torch.zeros((S, n, 4), dtype=torch.float32, device="cuda")
    s2 = torch.zeros((S, n), dtype=torch.float32, device="cuda")
    r.set_symbol_output(x4, s2)
    got, st_got = r.process(samples)
    assert torch.equal(got, ref)
    assert all(st_got[s]["bit_errors"] == st_ref[s]["bit_errors"] for s in range(S))
    assert torch.all(s2 > 0) and torch.all(torch.isfinite(x4))
    m = rx.Mlp(_params(13))
    r2 = receiver()
    r2.set_demapper(m)
    learned, st_l = r2.process(samples)
    c0, c1 = 4096, n - 512
    for s in range(S):
        want = m.infer(x4[s].contiguous(), s2[s].contiguous())
        assert torch.equal(learned[s], want), s
        hard = (learned[s, c0:c1].cpu().numpy() < 0).astype(np.uint8)
        assert st_l[s]["bit_errors"] == int(np.sum(hard != sts[s].bits[c0:c1])), s


def test_mlp_kernel_path_parameters_are_validated():
    """rx_mlp_set_param takes "train_tc" in {0, 1} and "infer" in {1, 2};
    other keys and values are refused and leave the setting unchanged."""
    rx = _rx()
    m = rx.Mlp(_params(21))
    assert m.get_param("train_tc") == 1 and m.get_param("infer") == 2
    for key, value in (("train_tc", 2), ("infer", 0), ("infer", 3), ("unknown", 1)):
        with pytest.raises(rx.RxError):
            m.set_param(key, value)
    assert m.get_param("train_tc") == 1 and m.get_param("infer") == 2
    m.set_param("infer", 1)
    assert m.get_param("infer") == 1
