"""Run the 2D cylinder workload (Mach-10 N2 past a half cylinder on a uniform
grid with cut cells) through the library and print one JSON line with the
particle counts, the status word, the counters and the device time per step.

    python -m paper_2508_05642_gb300.run_plane --steps 64 --nx 600 --ny 400

``--eager`` launches every kernel of every step separately instead of
replaying CUDA graphs (for per-kernel profilers)."""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs as I
from . import usp


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--nx", type=int, default=600)
    ap.add_argument("--ny", type=int, default=400)
    ap.add_argument("--ppc", type=float, default=30.0)
    ap.add_argument("--fp64", action="store_true", help="plain FP64 form (default FP32 state)")
    ap.add_argument("--eager", action="store_true", help="no CUDA graph replay")
    ap.add_argument("--seed", type=int, default=1)
    a = ap.parse_args(argv)
    w = I.cylinder_flow(seed=a.seed, nx=a.nx, ny=a.ny, ppc=a.ppc)
    dt = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.plane["n_inf"], w.plane["T_inf"])
    p = w.particles
    prec = usp.USP_FP64 if a.fp64 else usp.USP_FP32
    ctx = usp.usp_init_plane(w.species, w.plane, dt, w.area_frac, w.x, w.y, p.cx, p.cy, p.cz,
                             p.erot, p.lev, w.capacity, precision=prec, seed=a.seed,
                             use_graph=not a.eager)
    if a.warmup:
        usp.usp_step(ctx, a.warmup)
    usp.usp_sync(ctx)
    n0, _ = usp.usp_plane_count(ctx)
    t0 = time.perf_counter()
    usp.usp_step(ctx, a.steps)
    usp.usp_sync(ctx)
    el = time.perf_counter() - t0
    n1, nxt = usp.usp_plane_count(ctx)
    fl, cnt = usp.usp_status(ctx)
    print(json.dumps({"workload": w.name, "steps": a.steps, "warmup": a.warmup,
                      "precision": "f64" if a.fp64 else "f32", "graph": not a.eager,
                      "particles": [int(n0), int(n1)], "next_id": int(nxt),
                      "ms_per_step_host_clock": 1e3 * el / max(1, a.steps),
                      "particle_steps_per_s": 0.5 * (n0 + n1) * a.steps / el if el > 0 else None,
                      "flags": int(fl), "counters": [int(x) for x in np.asarray(cnt)]}))


if __name__ == "__main__":
    main()
