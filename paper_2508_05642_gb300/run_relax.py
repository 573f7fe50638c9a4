"""Homogeneous relaxation of viscous stress and heat flux (Sec. 5.A.1) through
the library: one cell of N2 at 4000 K sampled from Grad's 17-moment
distribution, stepped with the USP-FPM and the plain FPM method at several
time steps; prints one JSON line with the normalized L2 errors of the stress
and of the three heat fluxes against the model's analytic relaxation, and
the particle-steps per second of each run.

    python -m paper_2508_05642_gb300.run_relax --N 10000000

Analytic references (App. B, Eqs. analytic_sigma_full, analytic_qtr_full ..
analytic_qvib_full): sigma(t) = sigma(0) exp(-2 (1 - nu) t / tau) and
q(t) = q(0) exp(-3 t / tau) with tau = 2 mu (1 - nu) / p and
nu = 1 - 3 / (2 Pr), i.e. rates p / mu and Pr p / mu, at the initial state.
The error of a quantity is sqrt(sum (phi - phi_ref)^2) / sqrt(sum phi_ref^2)
over its three components and the states after every step up to t_end
(reading: the paper does not state its time window)."""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs as I
from . import usp

KB = 1.380649e-23


def _rates(sp: dict, n: float, T: float):
    """(p / mu, Pr) of the VSS gas at (n, T): mu from usp_tau_c and the VSS
    factor tau_c = c_a (5 - 2w)(7 - 2w) / (5 (c_a + 1)(c_a + 2)) mu / p, Pr of
    Eucken (Sec. 4.B) with the vibrational degrees of freedom at T."""
    ca, w = sp["c_alpha"], sp["omega"]
    f = ca * (5 - 2 * w) * (7 - 2 * w) / (5 * (ca + 1) * (ca + 2))
    p_over_mu = f / usp.usp_tau_c(sp, n, T)
    x = sp["theta_v"] / T
    xi = x / math.expm1(x)
    return p_over_mu, (14 + 2 * xi) / (19 + 2 * xi)


def _parts(mom):
    """off-diagonal stress and the three heat fluxes of a moments column"""
    return mom[10:13], mom[13:16], mom[16:19], mom[19:22]


def run(N=10_000_000, dts=(0.1, 0.5, 1.0, 2.0), t_end=8.0, precision=usp.USP_FP64, seed=1):
    base = I.stress_heat_flux_relaxation(seed=seed, N=N)
    sp = base.species
    n = float(base.ndens[0])
    T0 = float(base.T_nominal[0, 0])
    tau_c = usp.usp_tau_c(sp, n, T0)
    rate_s, pr = _rates(sp, n, T0)
    p = base.particles
    out = {"workload": base.name, "tau_c": tau_c, "t_end_over_tau_c": t_end,
           "precision": "f64" if precision == usp.USP_FP64 else "f32", "runs": {}}
    for method, name in ((usp.USP_METHOD_USP_FPM, "USP-FPM"), (usp.USP_METHOD_FPM, "FPM")):
        for r in dts:
            dt = r * tau_c
            steps = int(round(t_end / r))
            ctx = usp.usp_init_homogeneous(sp, base.offsets, base.ndens, np.array([dt]), p.cx,
                                           p.cy, p.cz, p.erot, p.lev, precision=precision,
                                           seed=seed, use_graph=False, method=method)
            m0 = usp.usp_moments(ctx)[:, 0]
            s0, qt0, qr0, qv0 = _parts(m0)
            num = np.zeros(4)
            den = np.zeros(4)
            t_run = 0.0
            for k in range(1, steps + 1):
                usp.usp_sync(ctx)
                t0 = time.perf_counter()
                usp.usp_step(ctx, 1)
                usp.usp_sync(ctx)
                t_run += time.perf_counter() - t0
                m = usp.usp_moments(ctx)[:, 0]
                t = k * dt
                refs = (s0 * math.exp(-rate_s * t), qt0 * math.exp(-pr * rate_s * t),
                        qr0 * math.exp(-pr * rate_s * t), qv0 * math.exp(-pr * rate_s * t))
                for i, (phi, ref) in enumerate(zip(_parts(m), refs)):
                    num[i] += float(((phi - ref) ** 2).sum())
                    den[i] += float((ref ** 2).sum())
            fl, _ = usp.usp_status(ctx)
            ctx.destroy()
            e = np.sqrt(num / den)
            out["runs"].setdefault(name, {})["%g" % r] = {
                "sigma": e[0], "q_tr": e[1], "q_rot": e[2], "q_vib": e[3], "steps": steps,
                "particle_steps_per_s": N * steps / t_run, "flags": int(fl)}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--N", type=int, default=10_000_000)
    ap.add_argument("--t-end", type=float, default=8.0, help="in units of tau_c")
    ap.add_argument("--fp32", action="store_true")
    ap.add_argument("--seed", type=int, default=1)
    a = ap.parse_args(argv)
    res = run(N=a.N, t_end=a.t_end, precision=usp.USP_FP32 if a.fp32 else usp.USP_FP64,
              seed=a.seed)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
