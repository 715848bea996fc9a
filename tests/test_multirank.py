"""The host side of several ranks (bench.py --gpus N), run as two gloo
processes on the CPU: each rank of the ensemble gets its own batch of
independent systems (rank 0 the reference one), single systems are
replicated, and the job's time is the slowest rank's while its units are
the sum over the ranks."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ens, _ = bench.rank_workload("ensemble_512", rank, world, nsys=6, n_lo=40, n_hi=80)
    disk, _ = bench.rank_workload("disk_260", rank, world)
    t = bench.max_over_ranks(1.5 + rank)
    u = bench.sum_over_ranks(ens.n_bodies)
    out.put((rank, t, u, ens.n_bodies, float(np.sum(ens.q)), float(np.sum(disk.q))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, u0, n0, e0, d0), (r1, t1, u1, n1, e1, d1) = res
    assert t0 == t1 == 2.5                    # the slowest rank's time
    assert u0 == u1 == n0 + n1                # units of all ranks
    assert e0 != e1                           # independent ensembles
    assert d0 == d1                           # replicated single system
    sys.path.insert(0, ROOT)
    import bench
    ref, _ = bench.rank_workload("ensemble_512", 0, 1, nsys=6, n_lo=40, n_hi=80)
    assert float(np.sum(ref.q)) == e0         # rank 0 keeps the reference batch
