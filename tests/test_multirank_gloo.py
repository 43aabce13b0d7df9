"""The host side of the multi-rank bench (replicas, no data-path collective) on
CPU: two gloo ranks draw independent point sets, meet at the barriers, and
agree on the slowest rank's time.  The GPU path runs the same helpers over
NCCL."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    import synth

    assert bench.dist_env() == (rank, world, rank)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench.WORKLOAD
        pts = synth.make_points(w["geometry"], n, bench.rank_seed(w["seed"], rank))
        assert pts.shape == (n, 3)
        # the ranks' inputs are independent draws of the same distribution
        mine = torch.tensor(pts.reshape(-1), dtype=torch.float64)
        other = [torch.zeros_like(mine) for _ in range(world)]
        tdist.all_gather(other, mine)
        assert not torch.equal(other[0], other[1])
        assert np.allclose(np.linalg.norm(other[1 - rank].numpy().reshape(n, 3), axis=1), 1.0)
        # max over ranks: every rank sees the slowest rank's time
        t = 0.25 + 0.5 * rank
        got = bench.max_over_ranks(t, world, tdist, torch.device("cpu"))
        assert got == 0.25 + 0.5 * (world - 1)
        tdist.barrier()
        assert bench.max_over_ranks(t, 1, tdist, torch.device("cpu")) == t
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks():
    mp.spawn(_rank_main, args=(2, _free_port(), 256), nprocs=2, join=True)


def test_rank_seeds_differ():
    import bench

    seeds = {bench.rank_seed(bench.WORKLOAD["seed"], r) for r in range(8)}
    assert len(seeds) == 8
