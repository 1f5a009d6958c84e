"""The multi-rank harness of bench.py on the host (gloo, world size 2): each
rank reads its place from the torchrun environment, draws its own streams
(weak scaling: the ranks' inputs differ and each is reproducible), the job's
time per step is the slowest rank's, and the reference arm runs on rank 0
alone (the other ranks return at once).  No GPU: the collective under test
is the max-reduce, on host tensors."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    assert bench.rank_env() == (rank, world, rank)
    assert bench.max_over_ranks(3.25) == 3.25          # no process group yet: the value itself
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(1.5 + rank)     # rank r's step takes 1.5 + r ms
        rx_a, bits_a = bench.make_inputs(rank, 512, 2)
        rx_b, bits_b = bench.make_inputs(rank, 512, 2)
        digests = [None] * world
        dist.all_gather_object(digests, (float(np.abs(rx_a).sum()), int(bits_a.sum())))

        class Args:
            ref_sym, warmup, steps = 1 << 10, 0, 1
        printed = None
        if rank != 0:
            import contextlib
            import io
            buf = io.StringIO()
            with contextlib.redirect_stdout(buf):
                ret = bench.run_reference(Args)
            printed = (ret, buf.getvalue())
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"slowest": slowest, "same_twice": bool(np.array_equal(rx_a, rx_b) and
                                                               np.array_equal(bits_a, bits_b)),
                       "digests": digests, "printed": printed}, f)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_streams_and_take_the_slowest_time(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["slowest"] == 2.5                      # the max over ranks, on every rank
        assert r["same_twice"]                          # each rank's inputs are reproducible
    d0, d1 = res[0]["digests"]
    assert d0 != d1                                     # the ranks draw different streams
    assert res[0]["digests"] == res[1]["digests"]
    assert res[1]["printed"] == [None, ""]              # the reference arm: rank 0 alone
