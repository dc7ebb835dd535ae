"""Multi-rank sharding on CPU (gloo, world size 2). Trajectories are
independent and their error draws depend only on (seed, trajectory id,
location), so contiguous id ranges per rank reproduce the single-rank
trajectories exactly; the only cross-rank operations are the sums of the
aggregates and the max of the elapsed times (as bench.py does under torchrun)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import montecarlo  # noqa: E402
from workloads import circuits as C  # noqa: E402

T, P, SEED = 240, 0.02, 7


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_range(rank, world, total):
    per = total // world
    return rank * per, per if rank < world - 1 else total - rank * per


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    circ = C.ghz(4)
    begin, n = _rank_range(rank, world, T)
    s, f, _ = montecarlo.run_trajectories(circ, SEED, begin, n, P / 3, P / 3, P / 3)
    sums = torch.tensor([s.sum(), (s * s).sum(), f.sum(), float(n)], dtype=torch.float64)
    dist.all_reduce(sums)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((sums.numpy().tolist(), float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_single_rank_aggregates():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    sums, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    s, f, _ = montecarlo.run_trajectories(C.ghz(4), SEED, 0, T, P / 3, P / 3, P / 3)
    assert sums[3] == T
    assert abs(sums[0] - s.sum()) < 1e-9 and abs(sums[1] - (s * s).sum()) < 1e-9
    assert sums[2] == f.sum()
    assert tmax == 2.0


def test_rank_ranges_partition_the_trajectories():
    for world in (1, 2, 3, 8):
        covered = []
        for r in range(world):
            b, n = _rank_range(r, world, 1001)
            covered += list(range(b, b + n))
        assert covered == list(range(1001))
