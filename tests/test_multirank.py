"""The multi-rank path of bench.py on CPU: two gloo ranks.  Each rank owns its
own independent instances (weak scaling, no collective on the data path);
the job's time is the slowest rank's, its particle count the sum; only rank 0
runs the reference arm."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    red = bench.RankReducer(dist, "cpu")
    w = bench.workload(rank, 0.002)
    n = w.n_particles
    t = 1.0 + rank          # a stand-in for the rank's timed region
    red.barrier()
    out[rank] = (red.max(t), red.sum(n), n, float(w.particles.cx[:64].sum()),
                 bench.run_reference(_RefArgs(), rank, world) if rank == 1 else 0)
    dist.destroy_process_group()


class _RefArgs:
    gpus, steps, warmup, scale = 2, 1, 0, 0.002


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 2.0                      # max over ranks
    assert r0[1] == r1[1] == r0[2] + r1[2]            # sum over ranks
    assert r0[3] != r1[3]                             # independent instances per rank
    assert r1[4] == 0                                 # reference arm: rank 1 exits without work


def test_single_process_reducer_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    red = bench.RankReducer()
    assert red.max(3.5) == 3.5 and red.sum(7) == 7.0
    red.barrier()
    assert bench.rank_seed(0) != bench.rank_seed(1)
