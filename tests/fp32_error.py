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
FP64 value for T_tr, T_rot, T_vib; sqrt(R T_tr) for U; R T_tr for the
viscous stress sigma_ij / rho = Pi_ij - delta_ij tr(Pi) / 3; (R T_tr)^1.5 for
the heat fluxes q / rho.  The table gives, over the first K steps and the six
instances, the root mean square (time-averaged L2) and the maximum.

  python tests/fp32_error.py [steps]      prints the table (needs a GPU)
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
           "T_vib": np.abs(g[6] - o[6]) / np.maximum(o[6], 1e-300)}

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


def markdown(table) -> str:
    ks = sorted(table)
    head = "| field | " + " | ".join(f"L2, {k} steps | max, {k} steps" for k in ks) + " |"
    sep = "|---|" + "---|---|" * len(ks)
    rows = [head, sep]
    for g in GROUPS:
        cells = []
        for k in ks:
            l2, mx = table[k][g]
            cells += [f"{l2:.2e}", f"{mx:.2e}"]
        rows.append(f"| {g} | " + " | ".join(cells) + " |")
    return "\n".join(rows)


if __name__ == "__main__":
    steps = int(sys.argv[1]) if len(sys.argv) > 1 else 200
    table, flags, sample, sizes = measure(steps, windows=(20, steps))
    print(f"instances {sample} with {sizes} particles; flags {flags:#x}")
    print(markdown(table))
    import json
    print(json.dumps({str(k): v for k, v in table.items()}))
