"""rx_unwrap_static: the unwrap stage for callers that may not allocate
device memory while they process (a real-time thread, or memory owned by
another allocator).  Its scratch is a static 64 KiB device array inside the
library.  The test checks it against rx_unwrap, which allocates its scratch,
over two calls in a row through the C ABI, and that an oversized request is
refused.  It sits in its own file so that it runs last in a full session and
also passes alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

B = 64


def _inputs(S, n, seed):
    rng = np.random.default_rng(seed)
    y = (rng.standard_normal((S, 2, n)) + 1j * rng.standard_normal((S, 2, n))).astype(np.complex64)
    steps = rng.integers(-2, 3, size=(S, n))
    b = (np.cumsum(steps, axis=1) + 32) % B            # a wandering phase index
    return torch.from_numpy(y).cuda(), torch.from_numpy(b.astype(np.uint8)).cuda()


def _run(r, fn, y, b, a, e, carry):
    S = y.shape[0]
    z = torch.zeros((S, 2, e - a), dtype=torch.complex64, device="cuda")
    pc = torch.zeros((S, e - a), dtype=torch.int16, device="cuda")
    cout = torch.zeros((S, 2), dtype=torch.int32, device="cuda")
    s2 = torch.zeros(S, dtype=torch.float64, device="cuda")
    fn(y, b, a, e, carry, z, pc, cout, s2)
    torch.cuda.synchronize()
    return z.cpu().numpy(), pc.cpu().numpy(), cout, s2.cpu().numpy()


def test_unwrap_static_matches_allocating_entry_point_twice():
    from paper_2108_07004_gb300 import rx
    S, n = 3, 9000
    r = rx.Receiver("gs4d64", taps=31, bps_phases=B, streams=S)
    y, b = _inputs(S, n, 7)
    carry = torch.tensor([[0, 32]] * S, dtype=torch.int32, device="cuda")
    # two consecutive ranges: the second starts from the first call's carry
    for a, e in ((0, 5000), (5000, n)):
        ref = _run(r, r.unwrap, y, b[:, a:e].contiguous(), a, e, carry)
        got = _run(r, r.unwrap_static, y, b[:, a:e].contiguous(), a, e, carry)
        scale = np.max(np.abs(ref[0]))
        assert np.max(np.abs(got[0] - ref[0])) <= 1e-5 * scale
        assert np.array_equal(got[1], ref[1])
        assert torch.equal(got[2], ref[2])
        assert np.allclose(got[3], ref[3], rtol=1e-12, atol=0)
        carry = ref[2]


def test_unwrap_static_refuses_more_scratch_than_it_has():
    """2048 streams x 10000 symbols: with one block per stream and wave
    (2048 streams already fill it) a block covers at most 4032 symbols, so a
    stream needs three blocks: 8 KiB of tickets + 24 KiB of increments +
    48 KiB of partial sums = 80 KiB > 64 KiB, and the call is refused before
    anything is launched.  Every buffer still has its full size, so nothing
    could be touched out of bounds either way."""
    from paper_2108_07004_gb300 import rx
    S, n = 2048, 10000
    r = rx.Receiver("gs4d64", taps=31, bps_phases=B, streams=S)
    y = torch.zeros((S, 2, n), dtype=torch.complex64, device="cuda")
    b = torch.full((S, n), 32, dtype=torch.uint8, device="cuda")
    carry = torch.tensor([[0, 32]] * S, dtype=torch.int32, device="cuda")
    z = torch.zeros((S, 2, n), dtype=torch.complex64, device="cuda")
    pc = torch.zeros((S, n), dtype=torch.int16, device="cuda")
    cout = torch.zeros((S, 2), dtype=torch.int32, device="cuda")
    s2 = torch.zeros(S, dtype=torch.float64, device="cuda")
    with pytest.raises(rx.RxError) as err:
        r.unwrap_static(y, b, 0, n, carry, z, pc, cout, s2)
    assert err.value.code == -1                          # RX_EINVAL
    assert "static" in str(err.value)
    torch.cuda.synchronize()
    assert int(cout.abs().sum()) == 0                    # nothing was written
