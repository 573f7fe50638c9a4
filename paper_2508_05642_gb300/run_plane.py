"""Run the 2D cylinder workload (Mach-10 N2 past a half cylinder on a grid
with cut cells, uniform or refined about the body) through the library and print one JSON line with the
particle counts, the status word, the counters and the device time per step.

    python -m paper_2508_05642_gb300.run_plane --steps 64 --nx 600 --ny 400

``--eager`` launches every kernel of every step separately instead of
replaying CUDA graphs (for per-kernel profilers).  ``--sample K`` runs K more
steps with the time averages on and adds the surface coefficients of the
cylinder (Sec. 5.C: C_f, C_h, pressure, total drag, peak heat flux)."""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs as I
from . import usp


def surface_coefficients(acc, plane: dict, species: dict, dt: float) -> dict:
    """Surface coefficients of the cylinder from the tallies of a sampled
    plane run (usp_sample_read layout): per polar-angle bin the wall stress
    and heat flux, C_f = tau / (rho U^2 / 2) and C_h = q / (rho U^3 / 2) with
    the freestream density and speed, the angle from the stagnation point
    (theta = 180 deg - phi on the upper half), the drag per unit length of
    the whole cylinder (twice the half body's, the lower half being the
    mirror image across the symmetry plane) and the peak heat flux."""
    ncell = usp.usp_plane_leaves(plane)
    steps = acc[ncell * 12]
    s = np.asarray(acc[ncell * 12 + 2:ncell * 12 + 2 + 4 * usp.USP_NSURF]).reshape(-1, 4)
    nb = len(s)
    m = species["m"]
    T = steps * dt
    r = plane["cyl_r"]
    dphi = 2 * math.pi / nb
    area = r * dphi * plane["depth"]
    phi = -math.pi + (np.arange(nb) + 0.5) * dphi
    fx = plane["F_num"] * m * s[:, 0] / T          # force on the wall per bin [N]
    fy = plane["F_num"] * m * s[:, 1] / T
    nxv, nyv = np.cos(phi), np.sin(phi)           # normal into the gas
    pressure = -(fx * nxv + fy * nyv) / area
    # shear along the surface, positive away from the stagnation point on the
    # upper half (direction of decreasing phi)
    tau = (fx * np.sin(phi) - fy * np.cos(phi)) / area
    q = plane["F_num"] * m * s[:, 2] / T / area
    rho = plane["n_inf"] * m
    U = plane["U_inf"]
    upper = (phi > 0) & (s[:, 3] > 0)
    theta = np.degrees(math.pi - phi[upper])
    order = np.argsort(theta)
    return {"sampled_steps": int(steps),
            "theta_deg": theta[order].tolist(),
            "C_f": (tau[upper] / (0.5 * rho * U * U))[order].tolist(),
            "C_h": (q[upper] / (0.5 * rho * U ** 3))[order].tolist(),
            "C_p": (pressure[upper] / (0.5 * rho * U * U))[order].tolist(),
            "drag_N_per_m": float(2.0 * fx.sum() / plane["depth"]),
            "peak_heat_flux_kW_per_m2": float(q[upper].max() / 1e3) if upper.any() else 0.0,
            "wall_events": int(s[:, 3].sum())}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--nx", type=int, default=600)
    ap.add_argument("--ny", type=int, default=400)
    ap.add_argument("--ppc", type=float, default=30.0)
    ap.add_argument("--fp64", action="store_true", help="plain FP64 form (default FP32 state)")
    ap.add_argument("--eager", action="store_true", help="no CUDA graph replay")
    ap.add_argument("--fpm", action="store_true",
                    help="the plain FPM method (cell values) instead of USP-FPM")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--sample", type=int, default=0, help="sampled steps after the timed ones")
    ap.add_argument("--case", choices=("mach10", "paper", "paper-refined"), default="mach10",
                    help="mach10: the 0.1 m cylinder benchmark grid (--nx/--ny/--ppc); paper: "
                         "the parameters of Sec. 5.C on its coarse Level 1 grid (--ppc); "
                         "paper-refined: the same with its Level 2 and Level 3 cells")
    a = ap.parse_args(argv)
    if a.case.startswith("paper"):
        w = I.cylinder_paper(seed=a.seed, ppc=a.ppc, refined=a.case == "paper-refined")
    else:
        w = I.cylinder_flow(seed=a.seed, nx=a.nx, ny=a.ny, ppc=a.ppc)
    dt = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.plane["n_inf"], w.plane["T_inf"])
    p = w.particles
    prec = usp.USP_FP64 if a.fp64 else usp.USP_FP32
    ctx = usp.usp_init_plane(w.species, w.plane, dt, w.area_frac, w.x, w.y, p.cx, p.cy, p.cz,
                             p.erot, p.lev, w.capacity, precision=prec, seed=a.seed,
                             use_graph=not a.eager,
                             method=usp.USP_METHOD_FPM if a.fpm else usp.USP_METHOD_USP_FPM)
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
    surf = None
    if a.sample > 0:
        usp.usp_sample(ctx, True)
        usp.usp_step(ctx, a.sample)
        surf = surface_coefficients(usp.usp_sample_read(ctx), w.plane, w.species, dt)
        fl, cnt = usp.usp_status(ctx)
    print(json.dumps({"workload": w.name, "method": "FPM" if a.fpm else "USP-FPM",
                      "steps": a.steps, "warmup": a.warmup,
                      "surface": surf,
                      "precision": "f64" if a.fp64 else "f32", "graph": not a.eager,
                      "particles": [int(n0), int(n1)], "next_id": int(nxt),
                      "ms_per_step_host_clock": 1e3 * el / max(1, a.steps),
                      "particle_steps_per_s": 0.5 * (n0 + n1) * a.steps / el if el > 0 else None,
                      "flags": int(fl), "counters": [int(x) for x in np.asarray(cnt)]}))


if __name__ == "__main__":
    main()
