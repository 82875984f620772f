"""The bench's multi-rank logic on CPU ranks (gloo, world size 2): the
whole-job time is the slowest rank's, the units are summed over ranks, and
an ensemble is split over ranks with every system on exactly one rank."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = [1.5, 2.25][rank]
    units = [1000.0, 3000.0][rank]
    t, u = bench.combine_ranks(t_local, units, world, "cpu")
    sizes = np.random.default_rng(4).integers(256, 65536, 301)
    a, b = bench.partition_systems(sizes, world)[rank]
    dist.barrier()
    q.put((rank, t, u, a, b))
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_and_split():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u, a, b in out:
        assert t == 2.25 and u == 4000.0  # slowest rank, summed units, on every rank
    (_, _, _, a0, b0), (_, _, _, a1, b1) = out
    assert a0 == 0 and b0 == a1 and b1 == 301  # contiguous, disjoint, complete


def test_partition_balances_tree_cost():
    import bench
    sizes = np.random.default_rng(9).integers(256, 65536, 4096)
    cost = sizes * np.log2(sizes)
    for world in (1, 2, 4, 8):
        parts = bench.partition_systems(sizes, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(sizes)
        assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
        share = np.array([cost[a:b].sum() for a, b in parts]) / cost.sum()
        assert np.all(np.abs(share - 1.0 / world) < 0.01)
    assert bench.combine_ranks(3.0, 7.0, 1, "cpu") == (3.0, 7.0)
