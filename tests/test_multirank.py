"""The multi-rank path of bench.py on CPU: two gloo ranks.  The ranks split
one population of 2 x 4096 instances by particle count (weak scaling, no
collective on the data path): together they hold every instance once, with
particle counts balanced to within the largest instance; each rank's
instances are exactly that part of the whole population.  The job's time is
the slowest rank's, its particle count the sum; only rank 0 runs the
reference arm."""
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
    w = bench.workload(rank, 0.002, world)
    n = w.n_particles
    t = 1.0 + rank          # a stand-in for the rank's timed region
    red.barrier()
    out[rank] = (red.max(t), red.sum(n), n, float(w.particles.cx[:64].sum()),
                 bench.run_reference(_RefArgs(), rank, world) if rank == 1 else 0,
                 list(map(int, w.extra["instances"])), w.offsets.copy(),
                 w.particles.cx.copy(), w.seed)
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
    assert r0[8] != r1[8]                             # independent Philox keys
    # the partition: disjoint, covering, balanced by particle count
    sys.path.insert(0, ROOT)
    from paper_2508_05642_gb300 import inputs as I
    import bench
    n_inst = 2 * bench.N_INST
    counts, _ = I.batched_parameters(seed=1, n_inst=n_inst, scale=0.002)
    i0, i1 = r0[5], r1[5]
    assert not set(i0) & set(i1) and sorted(i0 + i1) == list(range(n_inst))
    n0, n1 = int(counts[i0].sum()), int(counts[i1].sum())
    assert (n0, n1) == (r0[2], r1[2])
    assert abs(n0 - n1) <= counts.max()
    # each rank's particles are its instances of the one population
    whole = I.batched_instances(seed=1, n_inst=n_inst, scale=0.002)
    for idx, off, cx in ((i0, r0[6], r0[7]), (i1, r1[6], r1[7])):
        o = whole.offsets
        assert np.array_equal(cx, np.concatenate([whole.particles.cx[o[i]:o[i + 1]] for i in idx]))


def test_partition_balances_the_full_population():
    """At the benchmark's full size, 8 ranks: every instance once, per-rank
    particle counts within 1e-3 of the mean."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2508_05642_gb300 import inputs as I
    for world in (2, 4, 8):
        counts, _ = I.batched_parameters(seed=1, n_inst=world * bench.N_INST)
        parts = bench.partition(counts, world)
        assert sorted(i for p in parts for i in p) == list(range(len(counts)))
        tot = np.array([counts[p].sum() for p in parts], dtype=float)
        assert tot.max() / tot.mean() - 1.0 < 1e-3


def test_single_process_reducer_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    red = bench.RankReducer()
    assert red.max(3.5) == 3.5 and red.sum(7) == 7.0
    red.barrier()
    assert bench.rank_seed(0) != bench.rank_seed(1)
