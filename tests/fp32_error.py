"""Error of the FP32 form against the plain FP64 oracle on the batched workload.

The FP32 form keeps particle state and per-particle arithmetic in FP32 and
the cell sums, coefficients and conservation factors in FP64; the plain form
is FP64 throughout.  Both run the 4096-instance workload from the same
(float-exact) initial state with the same Philox streams; the FP32 run is the
library's (full size, autotuned, graph-replayed), the FP64 run is the CPU
oracle's plain form on six sampled instances -- the smallest, the largest and
four others -- each under its own cell index and particle ids.  Their paths
separate as rounding turns discrete outcomes (jump levels, +-1 picks) the
other way, so the error grows from rounding size into the sampling noise of
the instance.

Per reported field and step, the error is |FP32 - FP64| over a scale: the
FP64 value for T_tr, T_rot; T_tr for T_vib (which can be 0); sqrt(R T_tr)
for U; R T_tr for the
viscous stress sigma_ij / rho = Pi_ij - delta_ij tr(Pi) / 3; (R T_tr)^1.5 for
the heat fluxes q / rho.  The table gives, over the first K steps and the six
instances, the root mean square (time-averaged L2) and the maximum.

  python tests/fp32_error.py [batched|channel|plane]   prints a table (needs a GPU)

The channel (64 cells x 200 particles, 200 steps) and the cylinder plane
(600 x 400 cells, 6.9M particles, 20 steps: the oracle takes about a minute
per ten steps there) are measured the same way, per cell holding ten particles
or more, with N compared relatively.  In space, the two runs drift apart as
the flow amplifies rounding differences (about tenfold per 100 steps): cell
membership then differs, and the error grows into sampling noise.
"""
from __future__ import annotations

import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2508_05642_gb300 import inputs as I  # noqa: E402
from paper_2508_05642_gb300 import usp  # noqa: E402

GROUPS = ["U", "T_tr", "T_rot", "T_vib", "sigma", "q_tr", "q_rot", "q_vib"]


def sample_of(w):
    sizes = np.diff(w.offsets)
    return sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 1, 1000, 2048, 4095})


def _errors(g, o, R):
    """Normalised errors per group for moment vectors g, o (22, k)."""
    Ttr = o[4]
    vth = np.sqrt(R * Ttr)
    out = {"U": np.abs(g[1:4] - o[1:4]) / vth,
           "T_tr": np.abs(g[4] - o[4]) / o[4],
           "T_rot": np.abs(g[5] - o[5]) / o[5],
           "T_vib": np.abs(g[6] - o[6]) / Ttr}

    def sig(m):
        P = m[7:13].copy()
        tr = (P[0] + P[1] + P[2]) / 3.0
        P[0] -= tr; P[1] -= tr; P[2] -= tr
        return P
    out["sigma"] = np.abs(sig(g) - sig(o)) / (R * Ttr)
    for name, sl in (("q_tr", slice(13, 16)), ("q_rot", slice(16, 19)), ("q_vib", slice(19, 22))):
        out[name] = np.abs(g[sl] - o[sl]) / (R * Ttr) ** 1.5
    return out


def measure(steps: int = 200, windows=(20, 200)):
    w = I.batched_instances(seed=1, n_inst=4096, steps=steps)
    p = w.particles
    sample = sample_of(w)
    dt_g = np.array([w.dt_over_tau_c * usp.usp_tau_c(w.species, w.ndens[i], w.T_nominal[i, 0])
                     for i in range(w.n_cells)])
    ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt_g, p.cx, p.cy, p.cz, p.erot,
                                   p.lev, precision=usp.USP_FP32, seed=w.seed, use_graph=True)
    gm = np.zeros((steps, usp.USP_NMOM, len(sample)))
    for t in range(steps):
        usp.usp_step(ctx, 1)
        gm[t] = usp.usp_moments(ctx)[:, sample]
    flags, _ = usp.usp_status(ctx)
    ctx.destroy()
    # the oracle, plain FP64 form, on the sampled instances at their own
    # cell indices (the others empty) with their own particle ids
    sp = O.species(**w.species)
    dt_o = np.array([w.dt_over_tau_c * O.tau_c(sp, w.ndens[i], w.T_nominal[i, 0])
                     for i in range(w.n_cells)])
    p32 = p.astype_f32_exact()
    kmax = max(sample) + 1
    off = np.zeros(kmax + 1, dtype=np.int64)
    parts = []
    for k in range(kmax):
        n = int(w.offsets[k + 1] - w.offsets[k]) if k in sample else 0
        off[k + 1] = off[k] + n
        if n:
            b, e = int(w.offsets[k]), int(w.offsets[k + 1])
            parts.append((b, e))
    cat = lambda a: np.concatenate([a[b:e] for b, e in parts])  # noqa: E731
    pid = np.concatenate([np.arange(b, e, dtype=np.uint32) for b, e in parts])
    st = O.State.from_arrays(cat(p32.cx), cat(p32.cy), cat(p32.cz), cat(p32.erot), cat(p32.lev),
                             pid=pid)
    om = np.zeros_like(gm)
    for t in range(steps):
        O.homog_step(sp, 0, w.seed, t, 1, off, w.ndens[:kmax], dt_o[:kmax], st)
        om[t] = O.moments(sp, off, st)[:, sample]
    R = O.R(sp)
    table = {}
    for K in windows:
        errs = [_errors(gm[t], om[t], R) for t in range(K)]
        table[K] = {g: (float(math.sqrt(np.mean([np.mean(e[g] ** 2) for e in errs]))),
                        float(max(np.max(e[g]) for e in errs))) for g in GROUPS}
    return table, flags, sample, [int(x) for x in np.diff(w.offsets)[sample]]


def _spatial_table(gm, om, R, windows, nmin=10):
    """Errors of per-cell moment histories (steps, 22, cells) over the cells
    holding at least nmin particles in the FP64 run; N compared relatively."""
    table = {}
    for K in windows:
        errs = []
        for t in range(K):
            ok = om[t][0] >= nmin
            g, o = gm[t][:, ok], om[t][:, ok]
            e = _errors(g, o, R)
            e["N"] = np.abs(g[0] - o[0]) / o[0]
            errs.append(e)
        table[K] = {g: (float(math.sqrt(np.mean([np.mean(e[g] ** 2) for e in errs]))),
                        float(max(np.max(e[g]) for e in errs))) for g in ["N"] + GROUPS}
    return table


def measure_channel(steps: int = 200, windows=(20, 200)):
    """The Poiseuille workload (64 cells x 200 particles): the library's FP32
    run against the oracle's plain FP64 run, per cell and step."""
    w = I.channel_poiseuille(ny=64, ppc=200, steps=0)
    sp = O.species(**w.species)
    ch = O.channel(**w.channel)
    p = w.particles.astype_f32_exact()
    y = w.y.astype(np.float32).astype(np.float64)
    dto = w.dt_over_tau_c * O.tau_c(sp, w.n, w.channel["T_wall"])
    dtg = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.n, w.channel["T_wall"])
    st = O.ChannelState.from_arrays(y, p.cx, p.cy, p.cz, p.erot, p.lev)
    ctx = usp.usp_init_channel(w.species, w.channel, dtg, y, p.cx, p.cy, p.cz, p.erot, p.lev,
                               precision=usp.USP_FP32, seed=w.seed)
    gm = np.zeros((steps, usp.USP_NMOM, ch.ny))
    om = np.zeros_like(gm)
    for t in range(steps):
        usp.usp_step(ctx, 1)
        gm[t] = usp.usp_moments(ctx)
        off, _, _ = O.channel_step(sp, 0, w.seed, t, 1, ch, dto, st)
        om[t] = O.moments(sp, off, O.State.from_arrays(st.cx, st.cy, st.cz, st.erot, st.lev))
    flags, _ = usp.usp_status(ctx)
    ctx.destroy()
    return _spatial_table(gm, om, O.R(sp), windows), flags


def measure_plane(steps: int = 20, windows=(5, 20), nx=600, ny=400):
    """The Mach-10 cylinder (600 x 400 cells, 6.9M particles): the library's
    FP32 run against the oracle's plain FP64 run, per cell and step."""
    w = I.cylinder_flow(nx=nx, ny=ny, ppc=30)
    sp = O.species(**w.species)
    pl = O.plane(**w.plane)
    dto = w.dt_over_tau_c * O.tau_c(sp, w.plane["n_inf"], w.plane["T_inf"])
    dtg = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.plane["n_inf"], w.plane["T_inf"])
    q = w.particles
    arr = [a.astype(np.float32).astype(np.float64) for a in (w.x, w.y, q.cx, q.cy, q.cz, q.erot)]
    st = O.PlaneState(*arr, q.lev, w.capacity)
    ctx = usp.usp_init_plane(w.species, w.plane, dtg, w.area_frac, *arr, q.lev, w.capacity,
                             precision=usp.USP_FP32, seed=w.seed)
    ncell = pl.nx * pl.ny
    gm = np.zeros((steps, usp.USP_NMOM, ncell))
    om = np.zeros_like(gm)
    for t in range(steps):
        usp.usp_step(ctx, 1)
        gm[t] = usp.usp_moments(ctx)
        off, _, _ = O.plane_step(sp, 0, w.seed, t, 1, pl, w.area_frac, dto, st)
        n = st.n
        om[t] = O.moments(sp, off, O.State.from_arrays(st.cx[:n], st.cy[:n], st.cz[:n],
                                                       st.erot[:n], st.lev[:n]))
    flags, _ = usp.usp_status(ctx)
    ctx.destroy()
    return _spatial_table(gm, om, O.R(sp), windows), flags


def markdown(table) -> str:
    ks = sorted(table)
    head = "| field | " + " | ".join(f"L2, {k} steps | max, {k} steps" for k in ks) + " |"
    sep = "|---|" + "---|---|" * len(ks)
    rows = [head, sep]
    for g in table[ks[0]]:
        cells = []
        for k in ks:
            l2, mx = table[k][g]
            cells += [f"{l2:.2e}", f"{mx:.2e}"]
        rows.append(f"| {g} | " + " | ".join(cells) + " |")
    return "\n".join(rows)


if __name__ == "__main__":
    import json
    which = sys.argv[1] if len(sys.argv) > 1 else "batched"
    if which == "batched":
        table, flags, sample, sizes = measure(200, windows=(20, 200))
        print(f"batched: instances {sample} with {sizes} particles; flags {flags:#x}")
    elif which == "channel":
        table, flags = measure_channel(200, windows=(20, 200))
        print(f"channel 64 x 200: flags {flags:#x}")
    else:
        table, flags = measure_plane(20, windows=(5, 20))
        print(f"plane 600 x 400: flags {flags:#x}")
    print(markdown(table))
    print(json.dumps({str(k): v for k, v in table.items()}))
