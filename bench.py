#!/usr/bin/env python3
"""Benchmark of the batched homogeneous USP-FPM step on GB300.

Workload: 4096 independent single-cell N2 relaxation instances, particle
counts log-uniform in [1e3, 2e5] (~1.5e8 particles), T_tr ~ U[2000, 20000] K,
T_rot, T_vib ~ U[300, 3000] K, n = 1e23 m^-3, dt_i = 0.5 tau_c, FP32 particle
state with FP64 cell sums and coefficients.  Synthetic, seeded inputs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line is printed by rank 0.  ``value`` is particle-steps/s of the whole
job (all ranks: N GPUs share one population of N x 4096 instances, split by
particle count -- weak scaling, no collective on the data path), from CUDA
events on the library's stream with the
state resident in HBM.  ``e2e`` repeats the measurement through the C-ABI call
on pinned host buffers (state uploaded and moments read back every step).
``roofline`` rates the dominant kernel (the particle collide pass) against the
measured HBM copy bandwidth; ``cpu_baseline`` times the FP64 CPU oracle on a
bounded sample of the same workload.  ``--impl reference`` times that oracle
alone (the comparison arm).
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("particle-steps/s on 1 GB300 and % HBM roofline; FP32-batched vs plain FP64 form "
          "at stated error")
UNIT = "particle-steps/s"
N_INST = 4096
CPU_SAMPLE_INST = 64          # instances of the bounded oracle sample
# algorithmic bytes per particle-step: homogeneous cells read and write the
# state once (2 x 20 B FP32, 2 x 36 B FP64); the 2D plane path streams its
# 32-B FP32 state through the move/sort pass and the collide pass (4 x 32 B)
BYTES_PER_PARTICLE_STEP = {"f32": 40, "f64": 72, "plane_f32": 128}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink particle counts (debug only; the default is the full workload)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--late-steps", type=int, default=20,
                    help="steps timed from step 1000 on (0: skip)")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--fpm-steps", type=int, default=100,
                    help="steps of the plain FPM method (Sec. 2.C) on the same workload, FP32")
    ap.add_argument("--channel-steps", type=int, default=2000)
    ap.add_argument("--cylinder-steps", type=int, default=64)
    ap.add_argument("--refined-steps", type=int, default=64,
                    help="steps of the paper's cylinder on its three-level grid (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--variant", default=None,
                    help="force the FP32 particle-pass variant after autotuning: "
                         "'b2'..'b4' block-tiled or 'w2'..'w4' warp-tiled (for profiling a "
                         "given kernel on a smaller case)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampler running across the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        loaded = [x for x in sm if smax and x > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def source_hash():
    """Hash of the sources the batched collide kernel is compiled from."""
    h = hashlib.sha256()
    for f in ("usp_device.cuh", "usp_homog.cu"):
        h.update(open(os.path.join(ROOT, "paper_2508_05642_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(n_particles):
    """DRAM bytes per collide launch from the committed ncu summary, scaled to
    this launch's particle count; None if the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "collide_fp32_batched4096.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256_16") != source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_particle"]) * n_particles
    except (KeyError, ValueError):
        return None


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def rank_seed(rank):
    """Key of the Philox stream of a rank's instances: the ranks' streams are
    independent (particle ids are positions within a rank's arrays)."""
    return 1 + 1000 * rank


def partition(counts, world):
    """Instances of one workload split over ``world`` ranks by particle count
    (longest processing time first: the largest remaining instance goes to
    the rank with the fewest particles), each rank's list ascending.  With
    item sizes far below the per-rank total, the ranks' particle counts differ
    by less than the largest instance."""
    import heapq
    order = sorted(range(len(counts)), key=lambda i: (-int(counts[i]), i))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        tot, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (tot + int(counts[i]), r))
    return [sorted(p) for p in parts]


def workload(rank, scale, world=1):
    """The batched workload of a world of ``world`` ranks: one population of
    world x 4096 instances (weak scaling: the same particles per GPU on
    average at every world size), partitioned over the ranks by particle
    count with no collective; ``rank``'s share."""
    from paper_2508_05642_gb300 import inputs as I
    n_inst = N_INST * world
    counts, _ = I.batched_parameters(seed=1, n_inst=n_inst, scale=scale)
    mine = partition(counts, world)[rank]
    w = I.batched_instances(seed=1, n_inst=n_inst, steps=500, scale=scale,
                            select=None if world == 1 else mine)
    w.seed = rank_seed(rank)
    return w


class RankReducer:
    """Reductions of host scalars over the ranks of a process group (identity
    without one): the job's time is the slowest rank's, its particle count
    the sum over ranks."""

    def __init__(self, dist=None, device="cpu"):
        self.dist = dist
        self.device = device

    def _reduce(self, x, op):
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, self.dist.ReduceOp.MAX if self.dist else None)

    def sum(self, x):
        return self._reduce(x, self.dist.ReduceOp.SUM if self.dist else None)

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()


def fp32_error_table(m32, m64, species):
    """Per field, the root mean square and the maximum over the instances of
    |FP32 - FP64| over a scale (T_tr, T_rot: their value; T_vib: T_tr; U:
    sqrt(R T_tr); viscous stress / rho: R T_tr; heat fluxes / rho:
    (R T_tr)^1.5), both forms from the same state with the same draws."""
    import numpy as np
    R = 1.380649e-23 / species["m"]
    Ttr = m64[4]
    sig = lambda m: m[7:13] - np.concatenate([np.repeat(m[7:10].mean(axis=0, keepdims=True), 3, 0),  # noqa: E731
                                              np.zeros((3, m.shape[1]))])
    errs = {"U": np.abs(m32[1:4] - m64[1:4]) / np.sqrt(R * Ttr),
            "T_tr": np.abs(m32[4] - m64[4]) / Ttr, "T_rot": np.abs(m32[5] - m64[5]) / m64[5],
            "T_vib": np.abs(m32[6] - m64[6]) / Ttr,
            "sigma": np.abs(sig(m32) - sig(m64)) / (R * Ttr),
            "q_tr": np.abs(m32[13:16] - m64[13:16]) / (R * Ttr) ** 1.5,
            "q_rot": np.abs(m32[16:19] - m64[16:19]) / (R * Ttr) ** 1.5,
            "q_vib": np.abs(m32[19:22] - m64[19:22]) / (R * Ttr) ** 1.5}
    return {k: {"l2": float(np.sqrt(np.mean(v ** 2))), "max": float(np.max(v))}
            for k, v in errs.items()}


def config_of(w, steps, precision="f32"):
    return {"workload": w.name + (", FP32 state / FP64 cell sums" if precision == "f32"
                                  else ", FP64 plain"),
            "instances": w.n_cells, "particles_per_gpu": w.n_particles,
            "steps_timed": steps, "dt": "0.5 tau_c per instance",
            "l2": "inputs larger than L2 (state %.1f GB per GPU)" % (w.n_particles * 20 / 1e9),
            "parallelism": "one population of 4096 x N instances partitioned over the N GPUs by "
                           "particle count (weak scaling, no collective)"}


def cpu_baseline(w, target_s, fixed_steps=None):
    """Time the FP64 CPU oracle (as it stands) on the first CPU_SAMPLE_INST
    instances of the workload; returns (rate, cores, sample description)."""
    import numpy as np
    from oracle import oracle as O
    k = min(CPU_SAMPLE_INST, w.n_cells)
    off = w.offsets[:k + 1].copy()
    n = int(off[-1])
    p = w.particles
    st = O.State.from_arrays(p.cx[:n], p.cy[:n], p.cz[:n], p.erot[:n], p.lev[:n])
    sp = O.species(**w.species)
    dt = np.array([w.dt_over_tau_c * O.tau_c(sp, w.ndens[i], w.T_nominal[i, 0]) for i in range(k)])
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t0 = time.perf_counter()
    O.homog_step(sp, 1, w.seed, 0, 1, off, w.ndens[:k], dt, st)
    t1 = time.perf_counter() - t0
    steps = fixed_steps or max(1, min(500, int(target_s / max(t1, 1e-4))))
    t0 = time.perf_counter()
    O.homog_step(sp, 1, w.seed, 1, steps, off, w.ndens[:k], dt, st)
    el = time.perf_counter() - t0
    rate = n * steps / el
    return rate, cores, el, (f"first {k} of {w.n_cells} instances ({n} particles), {steps} steps, "
                             f"FP64 oracle (float-decision form), {el:.1f} s")


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    w = workload(0, args.scale)
    import numpy as np
    from oracle import oracle as O
    k = min(CPU_SAMPLE_INST, w.n_cells)
    off = w.offsets[:k + 1].copy()
    n = int(off[-1])
    p = w.particles
    st = O.State.from_arrays(p.cx[:n], p.cy[:n], p.cz[:n], p.erot[:n], p.lev[:n])
    sp = O.species(**w.species)
    dt = np.array([w.dt_over_tau_c * O.tau_c(sp, w.ndens[i], w.T_nominal[i, 0]) for i in range(k)])
    O.homog_step(sp, 1, w.seed, 0, args.warmup, off, w.ndens[:k], dt, st)
    t0 = time.perf_counter()
    O.homog_step(sp, 1, w.seed, args.warmup, args.steps, off, w.ndens[:k], dt, st)
    el = time.perf_counter() - t0
    rate = n * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"first {k} of {w.n_cells} instances ({n} particles) per step"
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, args.steps),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    from paper_2508_05642_gb300 import usp

    torch.cuda.set_device(local)
    usp.usp_select_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    red = RankReducer(dist, "cuda")
    barrier, max_over_ranks, sum_over_ranks = red.barrier, red.max, red.sum

    w = workload(rank, args.scale, world)
    dt = np.array([w.dt_over_tau_c * usp.usp_tau_c(w.species, w.ndens[i], w.T_nominal[i, 0])
                   for i in range(w.n_cells)])
    p = w.particles
    stream = torch.cuda.Stream()
    ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz, p.erot,
                                   p.lev, precision=usp.USP_FP32, seed=w.seed,
                                   stream=stream.cuda_stream, use_graph=True)
    N = w.n_particles
    if args.variant:
        usp.usp_set_variant(ctx, 1 if args.variant[0] == "w" else 0, int(args.variant[1:]))
    (warp_tiles, minb), tune_ms = usp.usp_tuning(ctx)
    usp.usp_step(ctx, args.warmup)
    # the state at the start of the timed region, kept on the device so that
    # the roofline pass below replays exactly the timed steps
    ckpt = torch.empty(usp.usp_checkpoint_bytes(ctx), dtype=torch.uint8, device="cuda")
    usp.usp_save(ctx, ckpt.data_ptr(), buf_is_device=True)
    torch.cuda.synchronize()

    # ---- timed region: K steps, graph replay, inputs resident in HBM ------
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = usp.usp_launch_count(ctx)
    e0.record(stream)
    usp.usp_step(ctx, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = usp.usp_launch_count(ctx) - l0
    ms = max_over_ranks(e0.elapsed_time(e1))
    total_particles = sum_over_ranks(float(N))
    value = total_particles * args.steps / (ms / 1e3)

    # ---- the same K steps again, from the checkpoint, with every kernel
    # bracketed by events (roofline); the FP32 form resumes bit for bit
    usp.usp_load(ctx, ckpt.data_ptr(), buf_is_device=True)
    del ckpt
    usp.usp_profile_enable(ctx, True)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    usp.usp_step(ctx, args.steps)
    f1.record(stream)
    kms, kn = usp.usp_profile_read(ctx)
    usp.usp_profile_enable(ctx, False)
    ms_prof = f0.elapsed_time(f1)
    collide_ms = kms[0] / max(1, kn[0])
    finalize_ms = kms[1] / max(1, kn[1])
    alg_bytes = BYTES_PER_PARTICLE_STEP["f32"] * N
    peak, peak_kind = hbm_peak()
    achieved = alg_bytes / (collide_ms / 1e3) / 1e9
    flags, counters = usp.usp_status(ctx)

    # ---- a late window: the cost grows as the levels heat up, so the rate
    # of steps 1000-1020 is reported beside that of the timed region
    late = None
    if args.late_steps > 0:
        done = args.warmup + args.steps
        start = max(done, 1000)
        usp.usp_step(ctx, start - done)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        usp.usp_step(ctx, args.late_steps)
        g1.record(stream)
        torch.cuda.synchronize()
        lms = max_over_ranks(g0.elapsed_time(g1))
        late = {"steps": f"{start}-{start + args.late_steps}",
                "value": total_particles * args.late_steps / (lms / 1e3), "unit": UNIT,
                "ms_per_step": lms / args.late_steps}

    # ---- end to end through the C ABI on pinned host buffers ---------------
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a, dt_: torch.from_numpy(np.ascontiguousarray(a, dtype=dt_)).pin_memory()
        hx, hy, hz, he = (pin(a, np.float32) for a in (p.cx, p.cy, p.cz, p.erot))
        hl = pin(p.lev, np.int32)
        mom = np.zeros((usp.USP_NMOM, w.n_cells))
        args_h = [hx.data_ptr(), hy.data_ptr(), hz.data_ptr(), he.data_ptr(), hl.data_ptr()]
        usp.usp_step_host(ctx, *args_h, 1, mom)     # warm-up of the path
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            usp.usp_step_host(ctx, *args_h, 1, mom)
        el = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": total_particles * args.e2e_steps / el, "unit": UNIT,
               "h2d_bytes_per_step": int(N * 20), "d2h_bytes_per_step": int(mom.nbytes),
               "ms_per_step": 1e3 * el / args.e2e_steps}
    ctx.destroy()
    del ctx

    # ---- the plain all-FP64 form on the same workload ----------------------
    fp64 = None
    if args.fp64_steps > 0:
        c64 = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz,
                                       p.erot, p.lev, precision=usp.USP_FP64, seed=w.seed,
                                       stream=stream.cuda_stream, use_graph=True)
        usp.usp_step(c64, 2)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        usp.usp_step(c64, args.fp64_steps)
        g1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(g0.elapsed_time(g1))
        fp64 = {"value": total_particles * args.fp64_steps / (ms64 / 1e3), "unit": UNIT,
                "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps}
        # the FP32 form's error against this FP64 run: a fresh FP32 context
        # (same state, same draws) stepped as far, every instance's moments
        m64 = usp.usp_moments(c64)
        c64.destroy()
        c32 = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz,
                                       p.erot, p.lev, precision=usp.USP_FP32, seed=w.seed,
                                       stream=stream.cuda_stream, use_graph=True,
                                       tile=1024)
        usp.usp_step(c32, 2 + args.fp64_steps)
        fp64["fp32_error"] = fp32_error_table(usp.usp_moments(c32), m64, w.species)
        fp64["fp32_error"]["steps"] = 2 + args.fp64_steps
        c32.destroy()

    # ---- the first-order FPM method on the same workload (FP32 state) -----
    fpm = None
    if args.fpm_steps > 0:
        cf = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz,
                                      p.erot, p.lev, precision=usp.USP_FP32, seed=w.seed,
                                      stream=stream.cuda_stream, use_graph=True,
                                      method=usp.USP_METHOD_FPM)
        usp.usp_step(cf, 3)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        usp.usp_step(cf, args.fpm_steps)
        g1.record(stream)
        torch.cuda.synchronize()
        msf = max_over_ranks(g0.elapsed_time(g1))
        ffl, _ = usp.usp_status(cf)
        fpm = {"method": "plain FPM (Gorji integrator, Milstein rotation, Gillespie levels)",
               "value": total_particles * args.fpm_steps / (msf / 1e3), "unit": UNIT,
               "ms_per_step": msf / args.fpm_steps, "steps": args.fpm_steps, "flags": int(ffl)}
        cf.destroy()

    # ---- the spatial path: force-driven Poiseuille channel (64 x 200) -----
    chan = None
    if args.channel_steps > 0:
        from paper_2508_05642_gb300 import inputs as I
        cw = I.channel_poiseuille(seed=rank_seed(rank))
        cdt = cw.dt_over_tau_c * usp.usp_tau_c(cw.species, cw.n, cw.channel["T_wall"])
        cp = cw.particles
        cctx = usp.usp_init_channel(cw.species, cw.channel, cdt, cw.y, cp.cx, cp.cy, cp.cz, cp.erot,
                                    cp.lev, precision=usp.USP_FP32, seed=cw.seed,
                                    stream=stream.cuda_stream, use_graph=True)
        usp.usp_step(cctx, 64)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        usp.usp_step(cctx, args.channel_steps)
        h1.record(stream)
        torch.cuda.synchronize()
        cms = max_over_ranks(h0.elapsed_time(h1))
        chan = {"workload": cw.name + ", FP32 state, reconstruction on",
                "value": sum_over_ranks(float(cw.n_particles)) * args.channel_steps / (cms / 1e3),
                "unit": UNIT, "ms_per_step": cms / args.channel_steps,
                "steps": args.channel_steps}
        cctx.destroy()

    # ---- the 2D path: Mach-10 cylinder, 600 x 400 cells, ~6.9M particles;
    # the paper's cylinder on its three-level grid, 422,730 cells, ~8.5M ----
    def plane_run(yw, steps, label):
        ydt = yw.dt_over_tau_c * usp.usp_tau_c(yw.species, yw.plane["n_inf"], yw.plane["T_inf"])
        yp = yw.particles
        yctx = usp.usp_init_plane(yw.species, yw.plane, ydt, yw.area_frac, yw.x, yw.y, yp.cx,
                                  yp.cy, yp.cz, yp.erot, yp.lev, yw.capacity,
                                  precision=usp.USP_FP32, seed=yw.seed,
                                  stream=stream.cuda_stream, use_graph=True)
        usp.usp_step(yctx, 16)
        torch.cuda.synchronize()
        n_a, _ = usp.usp_plane_count(yctx)
        l0 = usp.usp_launch_count(yctx)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        usp.usp_step(yctx, steps)
        q1.record(stream)
        torch.cuda.synchronize()
        yms = max_over_ranks(q0.elapsed_time(q1))
        n_b, _ = usp.usp_plane_count(yctx)
        yl = usp.usp_launch_count(yctx) - l0
        usp.usp_profile_enable(yctx, True)
        usp.usp_step(yctx, 8)
        pk, pn = usp.usp_profile_read(yctx)
        usp.usp_profile_enable(yctx, False)
        yfl, ycnt = usp.usp_status(yctx)
        # live count changes slowly; the mean of the two ends stands for it
        n_mean = 0.5 * (n_a + n_b)
        out = {"workload": yw.name + label,
               "value": sum_over_ranks(n_mean) * steps / (yms / 1e3), "unit": UNIT,
               "ms_per_step": yms / steps, "steps": steps, "cells": len(yw.area_frac),
               "first_step": 16, "particles": [int(n_a), int(n_b)], "gpu_launches": int(yl),
               "ms_per_step_particle_passes": pk[0] / 8, "ms_per_step_cell_passes": pk[1] / 8,
               "alg_bytes_per_particle_step": BYTES_PER_PARTICLE_STEP["plane_f32"],
               "flags": int(yfl)}
        yctx.destroy()
        return out

    cyl = None
    cyl_ref = None
    if args.cylinder_steps > 0 or args.refined_steps > 0:
        from paper_2508_05642_gb300 import inputs as I
    if args.cylinder_steps > 0:
        cyl = plane_run(I.cylinder_flow(seed=rank_seed(rank)), args.cylinder_steps,
                        ", FP32 state, reconstruction on, dt = 0.5 tau_c")
    if args.refined_steps > 0:
        cyl_ref = plane_run(I.cylinder_paper(seed=rank_seed(rank), refined=True),
                            args.refined_steps, ", FP32 state, reconstruction on")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, cores, el, sample = cpu_baseline(w, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": config_of(w, args.steps),
                "gpu_launches": int(launches),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_source": peak_kind,
                             "traffic": profiled_traffic(N),
                             "kernel": ("collide_warp_kernel<float>" if warp_tiles
                                        else "collide_kernel<float>"),
                             "kernel_ms": collide_ms, "alg_bytes_per_launch": alg_bytes,
                             "finalize_ms": finalize_ms, "ms_per_step_profiled": ms_prof / args.steps,
                             "autotune": {"warp_tiles": warp_tiles, "blocks_per_sm": minb,
                                          "ms_block_tiled_2_3_4": [float(x) for x in tune_ms[:3]],
                                          "ms_warp_tiled_2_3_4": [float(x) for x in tune_ms[3:]]}},
                "late_window": late,
                "e2e": e2e, "cpu_baseline": cpu, "fp64_plain": fp64, "fpm_method": fpm,
                "poiseuille_channel": chan,
                "cylinder_plane": cyl, "cylinder_plane_refined": cyl_ref,
                "clocks": clk,
                "status": {"flags": int(flags), "counters": [int(x) for x in counters]}}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
