"""Pins of the oracle's plain FPM method (Sec. 2.B model, Sec. 2.C particle
scheme): Gillespie's direct method against the exact transient distribution of
the master equation's linear birth-death process (matrix exponential of its
generator), the model's relaxation rates against viscosity and Prandtl
number, the conservation targets against the Landau-Teller equations of
Sec. 2.A, and one full particle step against the moment relaxation the scheme
implies (App. A: stress with exp(-2 dt/tau) + nu (1 - exp(-2 dt/tau)), heat
fluxes with exp(-3 dt/tau)).  No test re-types the oracle's formulas."""
import math

import numpy as np
import pytest
from scipy import linalg, stats

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I

KB = 1.380649e-23


def _sp(**over):
    d = I.n2_vhs_relaxation_species()
    d.update(over)
    return O.species(**d)


def _exact_levels(I0, lam_up, lam_dn, K=80):
    """Distribution of the level after one step (time 1 in units of dt) of the
    birth-death process with rates lam_up (I+1) up and lam_dn I down."""
    Q = np.zeros((K, K))
    for i in range(K):
        up = lam_up * (i + 1) if i + 1 < K else 0.0
        dn = lam_dn * i
        if i + 1 < K:
            Q[i, i + 1] = up
        if i > 0:
            Q[i, i - 1] = dn
        Q[i, i] = -(up + dn)
    return linalg.expm(Q)[I0]


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("I0,lam_up,lam_dn", [(0, 0.3, 1.1), (3, 0.05, 0.45), (6, 0.8, 1.9)])
def test_gillespie_matches_exact_transient_distribution(form, I0, lam_up, lam_dn):
    """Sec. 2.C: Gillespie's direct method samples the master equation
    exactly; the sampled levels after one step follow exp(Q) of its generator."""
    n = 60000
    levels = np.array([O.gillespie(I0, lam_up, lam_dn, 11, pid, 3, form)[0] for pid in range(n)])
    p = _exact_levels(I0, lam_up, lam_dn)
    counts = np.bincount(levels, minlength=len(p))[:len(p)]
    assert counts.sum() == n
    exp = p * n
    # pool the sparse tail into one bin
    keep = exp >= 10
    obs = np.append(counts[keep], n - counts[keep].sum())
    ex = np.append(exp[keep], n - exp[keep].sum())
    _, pval = stats.chisquare(obs, ex)
    assert pval > 1e-4, (pval, obs, ex)
    # mean level: relaxation toward lam_up / (lam_dn - lam_up) at rate lam_dn - lam_up
    eb = lam_up / (lam_dn - lam_up)
    mean = eb + (I0 - eb) * math.exp(-(lam_dn - lam_up))
    assert abs(levels.mean() - mean) < 5 * levels.std() / math.sqrt(n)


def test_gillespie_without_rates_keeps_the_level():
    assert O.gillespie(0, 0.0, 0.7, 1, 2, 3)[0] == 0
    assert O.gillespie(4, 0.0, 0.0, 1, 2, 3)[0] == 4


def test_fpm_relaxation_rates_give_viscosity_and_prandtl():
    """Sec. 2.B: the FPM model relaxes stress at p/mu (the viscosity it is
    built for, mu of Sec. 4.A) and heat fluxes at Pr p/mu (its Prandtl
    number, Eucken's Pr of Sec. 4.B); the scheme's per-step factors of App. A
    tend to those rates as dt -> 0."""
    sp = _sp()
    n, T = 1e23, 3000.0
    for Tv in (800.0, 3000.0):
        p = n * KB * T
        fc = O.fpm_coeffs(sp, n, 1e-14, T, T, Tv)
        mu = fc.mu   # Bird's VHS viscosity, pinned in test_oracle_pins
        a2 = fc.alpha ** 2
        rate_sigma = -math.log(a2 + fc.nu * (1.0 - a2)) / fc.dt
        rate_q = -3.0 * math.log(fc.alpha) / fc.dt
        assert rate_sigma == pytest.approx(p / mu, rel=1e-5)
        x = sp.theta_v / Tv
        xi = x / math.expm1(x)
        pr_eucken = (14 + 2 * xi) / (19 + 2 * xi)
        assert rate_q / rate_sigma == pytest.approx(pr_eucken, rel=1e-5)


def test_fpm_targets_follow_landau_teller():
    """Sec. 2.A: de_rot/dt = (e_rot(T_tr) - e_rot(T_rot))/tau_rot and
    de_vib/dt = (e_vib(T_tr) - e_vib(T_vib))/tau_vib; the FPM targets after
    a small dt change the mode energies by dt times those rates, with an
    O(dt^2) remainder."""
    sp = _sp(Z_rot=5.0, Z_vib=20.0)
    R = O.R(sp)
    n, Ttr, Trot, Tvib = 1e23, 6000.0, 1500.0, 900.0
    tau_c = O.tau_c(sp, n, Ttr)
    def ev(T):
        return R * sp.theta_v / math.expm1(sp.theta_v / T)
    errs = []
    for k in (1e-3, 1e-4):
        dt = k * tau_c
        fc = O.fpm_coeffs(sp, n, dt, Ttr, Trot, Tvib)
        drot = (R * Ttr - R * Trot) / (5.0 * tau_c) * dt
        dvib = (ev(Ttr) - ev(Tvib)) / (20.0 * tau_c) * dt
        e_rot_err = (fc.e_rot_tgt - R * Trot) / drot - 1.0
        e_vib_err = (fc.e_vib_tgt - ev(Tvib)) / dvib - 1.0
        errs.append((abs(e_rot_err), abs(e_vib_err)))
        assert abs(e_rot_err) < 10 * k and abs(e_vib_err) < 10 * k
    # first-order remainder: ten times smaller dt, ten times smaller error
    assert errs[1][0] < 0.2 * errs[0][0] and errs[1][1] < 0.2 * errs[0][1]


def _skewed_state(rng, N, sp, T=4000.0):
    R = O.R(sp)
    s = math.sqrt(R * T)
    g = rng.standard_normal((N, 3))
    cx = s * (g[:, 0] + 0.25 * (g[:, 0] ** 2 - 1))
    cy = s * 1.2 * g[:, 1]
    cz = s * 0.8 * g[:, 2] + 0.3 * s * g[:, 1]
    w = 1 + 0.8 * np.tanh(g[:, 0])
    erot = rng.exponential(R * T, N) * w
    x = math.exp(-sp.theta_v / T)
    lev = (rng.geometric(1 - x, N) - 1) * (1 + (g[:, 0] > 0.5)).astype(np.int32)
    return O.State.from_arrays(cx, cy, cz, erot, lev.astype(np.int32))


def _sigma_q(m):
    Pi = m[7:13, 0]
    tr = Pi[:3].sum() / 3
    sig = np.concatenate([Pi[:3] - tr, Pi[3:]])
    return sig, m[13:16, 0], m[16:19, 0], m[19:22, 0]


@pytest.mark.parametrize("form", [0, 1])
def test_fpm_one_step_stress_and_heat_flux_relaxation(form):
    """One full FPM step including the conservation scheme: the stress
    follows alpha^2 + nu (1 - alpha^2) and all three heat fluxes alpha^3
    (alpha = exp(-dt/tau)), in expectation: the moment relaxation the
    scheme of Sec. 2.C implies (App. A)."""
    sp = _sp(Z_rot=5.0, Z_vib=10.0)
    rng = np.random.default_rng(40 + form)
    N = 400000
    st = _skewed_state(rng, N, sp)
    off = [0, N]
    m0 = O.moments(sp, off, st)
    n = 1e23
    dt = 0.5 * O.tau_c(sp, n, m0[4, 0])
    fc = O.fpm_coeffs(sp, n, dt, m0[4, 0], m0[5, 0], m0[6, 0])
    fl, cnt = O.homog_step_fpm(sp, form, 5, 0, 1, off, [n], [dt], st)
    assert fl == 0 and cnt[O.C_CHOL_FIX] == 0
    m1 = O.moments(sp, off, st)
    s0, qt0, qr0, qv0 = _sigma_q(m0)
    s1, qt1, qr1, qv1 = _sigma_q(m1)
    R = O.R(sp)
    T = m0[4, 0]
    a = fc.alpha
    ss = R * T * math.sqrt(2.0 / N) * 4
    assert np.allclose(s1, (a * a + fc.nu * (1 - a * a)) * s0, atol=ss)
    assert np.abs(s0).max() > 20 * ss
    qs = (R * T) ** 1.5 * math.sqrt(15.0 / N) * 4
    assert np.allclose(qt1, a ** 3 * qt0, atol=qs)
    assert np.allclose(qr1, a ** 3 * qr0, atol=qs)
    qvs = (R * T) * math.sqrt(R * T) * math.sqrt(12.0 / N) * 4
    assert np.allclose(qv1, a ** 3 * qv0, atol=qvs)
    assert np.abs(qt0).max() > 10 * qs and np.abs(qr0).max() > 8 * qs


def test_fpm_conservation_per_cell_is_exact():
    """Sec. 4.C with the FPM method: momentum and total energy of each cell
    are conserved to FP64 rounding while the modes exchange energy."""
    sp = _sp()
    w = I.batched_instances(seed=3, n_inst=6, nmin=50, nmax=3000, steps=0)
    st = O.State.from_arrays(w.particles.cx, w.particles.cy, w.particles.cz,
                             w.particles.erot, w.particles.lev)
    R = O.R(sp)
    Rth = R * sp.theta_v
    dt = np.array([0.5 * O.tau_c(sp, w.ndens[i], w.T_nominal[i, 0]) for i in range(w.n_cells)])
    def totals():
        out = []
        for i in range(w.n_cells):
            b, e = w.offsets[i], w.offsets[i + 1]
            mom = np.array([st.cx[b:e].sum(), st.cy[b:e].sum(), st.cz[b:e].sum()])
            en = 0.5 * (st.cx[b:e] ** 2 + st.cy[b:e] ** 2 + st.cz[b:e] ** 2).sum() \
                + st.erot[b:e].sum() + Rth * st.lev[b:e].sum()
            out.append((mom, en))
        return out
    t0 = totals()
    e_rot0 = [st.erot[w.offsets[i]:w.offsets[i + 1]].mean() for i in range(w.n_cells)]
    fl, _ = O.homog_step_fpm(sp, 0, 9, 0, 1, w.offsets, w.ndens, dt, st)
    assert fl & ~O.F_TREL_CLAMP == 0
    t1 = totals()
    for (m0, e0), (m1, e1) in zip(t0, t1):
        scale = math.sqrt(2 * e0 / 1.0)
        assert np.all(np.abs(m1 - m0) <= 1e-12 * scale * 1e3)
        assert abs(e1 - e0) <= 1e-12 * e0
    e_rot1 = [st.erot[w.offsets[i]:w.offsets[i + 1]].mean() for i in range(w.n_cells)]
    assert any(abs(a - b) > 1e-3 * a for a, b in zip(e_rot0, e_rot1))
