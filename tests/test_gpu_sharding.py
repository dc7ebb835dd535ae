"""The library's trajectory-range split in two processes (gloo, world size 2)
on one GPU, as bench.py shards trajectories under torchrun: each rank samples
and runs its contiguous range of trajectory ids through the C ABI; the ranks'
per-trajectory scores, gathered over gloo, equal one process's run of the
whole range bit for bit, and the summed aggregates agree. The two processes
launch independent kernels (no kernel waits on the other process)."""
import os
import socket

import numpy as np
import pytest

from workloads import circuits as C

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

pytestmark = pytest.mark.gpu

T, P, SEED = 400, 4e-3, 5
CASES = {"resident": (lambda: C.qaoa_maxcut(12, 4), {}),
         "streaming": (lambda: C.brickwork(16, 12, 3), {"tile_qubits": 12})}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_range(rank, world, total):
    per = total // world
    return rank * per, per if rank < world - 1 else total - rank * per


def _scores(case, begin, n):
    from paper_2301_07264_gb300 import arso
    make, kw = CASES[case]
    circ = make()
    cc = arso.compile_circuit(circ.n, circ.gates, **kw)
    errs = arso.sample_errors(cc, P / 3, P / 3, P / 3, SEED, begin, n)
    s = np.zeros(n)
    f = np.zeros(n, dtype=np.uint8)
    arso.run_trajectories(cc, errs, circ.criterion, s, f)
    return s, f


def _worker(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    begin, n = _rank_range(rank, world, T)
    s, f = _scores(case, begin, n)
    parts = [torch.zeros(_rank_range(r, world, T)[1], dtype=torch.float64) for r in range(world)]
    dist.all_gather(parts, torch.from_numpy(s))
    sums = torch.tensor([s.sum(), (s * s).sum(), float(f.sum()), float(n)], dtype=torch.float64)
    dist.all_reduce(sums)
    if rank == 0:
        out.put((torch.cat(parts).numpy(), sums.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_two_ranks_on_the_library_reproduce_one_process(case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, sums = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    s, f = _scores(case, 0, T)
    assert np.array_equal(gathered, s)
    assert sums[3] == T and sums[2] == f.sum()
    assert abs(sums[0] - s.sum()) < 1e-9 and abs(sums[1] - (s * s).sum()) < 1e-9
