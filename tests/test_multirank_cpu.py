"""The multi-rank (N > 1) host logic of bench.py on CPU with two gloo ranks.

Each rank solves its own batch of rhs (independent sources, no data-path
collective); the job's time is the maximum over ranks and the throughput sums
every rank's work over that time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import synthetic as syn
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = 1.0 + rank          # rank 1 is the slower one
    t = bench.allreduce_max(world, t_local, device="cpu")
    seed = bench.rank_rhs_seed(1001, rank)
    b = syn.gaussian_spinors((2, 2, 2, 2), 1, seed)
    first = torch.tensor([b.real.ravel()[0]], dtype=torch.float64)
    gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, first)
    value = bench.aggregate_throughput(world, 100.0, 3, t)
    out[rank] = (t, seed, [float(g) for g in gathered], value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_host_logic():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    (t0, s0, g0, v0), (t1, s1, g1, v1) = out[0], out[1]
    assert t0 == t1 == 2.0                       # max over ranks
    assert s0 != s1 and g0[0] != g0[1]           # distinct rhs batches per rank
    assert v0 == v1 == pytest.approx(2 * 100.0 * 3 / 2.0)
