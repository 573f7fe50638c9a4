"""The Grad-17 initial state of the stress / heat-flux relaxation (Sec. 5.A.1):
its moments, measured by the oracle's moment definitions, carry the imposed
stress and heat fluxes at T_eq (the acceptance sampler clamps the weight in the
far tails, so the heat fluxes come out a few per cent low)."""
import math

import numpy as np

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I


def test_grad17_moments():
    sp = I.n2_vss_species(10.0, 50.0)
    rng = np.random.default_rng(3)
    N = 1500000
    p = I.grad17_particles(rng, N, sp["m"], sp["theta_v"], 4000.0)
    assert len(p.cx) == N
    osp = O.species(**sp)
    m = O.moments(osp, [0, N], O.State.from_arrays(p.cx, p.cy, p.cz, p.erot, p.lev))[:, 0]
    RT = O.R(osp) * 4000.0
    for f in (4, 5, 6):
        assert abs(m[f] / 4000.0 - 1) < 0.01
    assert np.all(np.abs(m[10:13] / RT - 0.1) < 0.006)          # off-diagonal stress
    dev = m[7:10] - m[7:10].mean()
    assert np.all(np.abs(dev / RT) < 0.006)                      # no normal stress
    # statistical error of a component: 0.0024 (RT)^1.5 (q_tr), less for the others
    for q in (m[13:16], m[16:19], m[19:22]):
        assert np.all(np.abs(q / RT ** 1.5 - 0.1) < 0.015)


def test_stress_heat_flux_workload_matches_printed_set_up():
    w = I.stress_heat_flux_relaxation(N=1000, dt_over_tau_c=0.5)
    assert w.n_particles == 1000 and w.steps == 16
    assert w.ndens[0] == 1e24 and tuple(w.T_nominal[0]) == (4000.0, 4000.0, 4000.0)
    assert w.species["Z_rot"] == 10.0 and w.species["Z_vib"] == 50.0
    osp = O.species(**w.species)
    # the printed mean collision time of Sec. 5.A.1
    assert abs(O.tau_c(osp, 1e24, 4000.0) / 1.4573e-9 - 1) < 2e-3
