"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test names the passage of Kim & Jun (arXiv 2508.05642) or the textbook
fact it checks.  None of them re-types the oracle's own formula: they use
published known answers, printed values, closed forms of the method's moment
relaxations (Sec. 3.A), the Taylor expansions of App. B, library routines
(scipy) and exact distributional identities.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KB = 1.380649e-23


def _sp(**over):
    d = I.n2_vhs_relaxation_species()
    d.update(over)
    return O.species(**d)


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# random numbers
# --------------------------------------------------------------------------
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (SC'11)."""
    for row in _read_table("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        assert O.philox(v[0:4], v[4:6]) == tuple(v[6:10])


def test_uniform_maps_are_open_and_exact():
    # form 0: (x + 0.5) 2^-32; form 1: (2 (x >> 9) + 1) 2^-24
    assert O.uniform(0, 0) == 2.0 ** -33
    assert O.uniform(0xFFFFFFFF, 0) == 1.0 - 2.0 ** -33
    assert O.uniform(0, 1) == 2.0 ** -24
    assert O.uniform(0xFFFFFFFF, 1) == 1.0 - 2.0 ** -24
    assert np.float32(O.uniform(0x12345678, 1)) == O.uniform(0x12345678, 1)
    xs = np.random.default_rng(3).integers(0, 2 ** 32, 2000, dtype=np.uint64)
    for x in xs[:200]:
        u0, u1 = O.uniform(int(x), 0), O.uniform(int(x), 1)
        assert 0.0 < u0 < 1.0 and 0.0 < u1 < 1.0 and abs(u0 - u1) < 2.0 ** -23


def test_philox_stream_uniformity():
    """Words of consecutive counters are uniform (chi^2 on 64 bins)."""
    words = []
    for c in range(4000):
        words.extend(O.philox([c, 7, 0, 0], [1, 0]))
    u = (np.array(words, dtype=np.float64) + 0.5) / 2 ** 32
    h, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2 = ((h - len(u) / 64) ** 2 / (len(u) / 64)).sum()
    assert stats.chi2.sf(chi2, 63) > 1e-4


# --------------------------------------------------------------------------
# closed-form physics (Sec. 2.A, 4.A, 4.B)
# --------------------------------------------------------------------------
def test_cv_vib_is_derivative_of_e_vib():
    """c_v,vib = d e_vib/dT (Sec. 2.A definition); the printed formula lacks the
    square on sinh, the derivative pins the squared form."""
    sp = _sp()
    for T in [150.0, 300.0, 1000.0, 3371.0, 8000.0, 30000.0]:
        h = T * 1e-5
        fd = (O.e_vib(sp, T + h) - O.e_vib(sp, T - h)) / (2 * h)
        assert O.cv_vib(sp, T) == pytest.approx(fd, rel=1e-7)
    # high-T limit of a harmonic oscillator: c_v -> R
    assert O.cv_vib(sp, 1e7) == pytest.approx(O.R(sp), rel=1e-6)
    assert O.cv_vib(sp, 0.0) == 0.0 and O.e_vib(sp, 0.0) == 0.0


def test_T_vib_inverts_e_vib():
    sp = _sp()
    Rth = O.R(sp) * sp.theta_v
    for T in [100.0, 300.0, 2000.0, 20000.0]:
        ebar = O.e_vib(sp, T) / Rth
        assert O.T_vib_from_mean_level(sp, ebar) == pytest.approx(T, rel=1e-12)
    assert O.T_vib_from_mean_level(sp, 0.0) == 0.0


def test_tau_c_printed_values():
    """Printed mean collision times of Sec. 5.A.1 and 5.A.2 (VSS N2)."""
    sp = O.species(**I.n2_vss_species())
    for n, T, tau, tol in _read_table("tau_c_printed.txt"):
        assert O.tau_c(sp, float(n), float(T)) == pytest.approx(float(tau), rel=float(tol))
    # the molecular mass printed in Sec. 5 (6.63e-26 kg) does not reproduce them
    bad = O.species(**dict(I.n2_vss_species(), m=6.63e-26))
    assert abs(O.tau_c(bad, 1e24, 6000.0) / 1.3132e-9 - 1) > 0.1


def test_vhs_viscosity_is_birds_formula():
    """With c_alpha = 1 the VSS reference viscosity is Bird's VHS formula
    mu_ref = 15 sqrt(pi m k T_ref) / (2 pi d^2 (5 - 2w)(7 - 2w))."""
    sp = _sp()
    w, d, m, Tr = sp.omega, sp.d_ref, sp.m, sp.T_ref
    mu_ref = 15 * math.sqrt(math.pi * m * KB * Tr) / (2 * math.pi * d * d * (5 - 2 * w) * (7 - 2 * w))
    assert O.mu(sp, Tr) == pytest.approx(mu_ref, rel=1e-14)
    assert O.mu(sp, 4 * Tr) == pytest.approx(mu_ref * 4 ** w, rel=1e-13)


def test_eucken_limits():
    sp = _sp()
    assert O.prandtl(sp, 0.0) == pytest.approx(14 / 19)          # frozen vibration
    assert O.prandtl(sp, 1e9) == pytest.approx(16 / 21, rel=1e-6)  # xi -> 1


def test_parker_and_millikan_white_numbers():
    """Sec. 5.C collision numbers: Parker tends to Z_rot_inf at high T."""
    d = I.n2_vss_species()
    d.update(zmodel=1, Zrot_inf=23.0, T_star=91.5, C1=9.1, C2=220.0, sigma_vib=5.81e-21,
             T_ref=290.0, omega=0.70, c_alpha=1.0)
    sp = O.species(**d)
    zr, zv = O.collision_numbers(sp, 1e12)
    assert zr == pytest.approx(23.0, rel=1e-4)
    zr1, zv1 = O.collision_numbers(sp, 1000.0)
    r = 91.5 / 1000.0
    assert zr1 == pytest.approx(23.0 / (1 + math.pi ** 1.5 / 2 * math.sqrt(r) + (math.pi + math.pi ** 2 / 4) * r))
    assert zv1 > 0 and zv > 0


# --------------------------------------------------------------------------
# per-cell coefficients (Sec. 3.A)
# --------------------------------------------------------------------------
def _coeffs(sp, T_tr, T_rot, T_vib, dt_over_tauc=0.5, n=1e23):
    dt = dt_over_tauc * O.tau_c(sp, n, T_tr)
    return O.cell_coeffs(sp, n, dt, T_tr, T_rot, T_vib)


def test_alpha_nu_reproduce_sigma_and_q_relaxation():
    """Eqs. USP-FPM_alpha_tr / USP-FPM_nu make the particle scheme's stress
    factor alpha^2 + nu (1 - alpha^2) equal Eq. sigma_relax and its heat-flux
    factor alpha^3 equal Eq. qtr_relax."""
    sp = _sp()
    for T in [(10000, 300, 300), (2000, 3000, 2500), (6000, 4000, 2000)]:
        c = _coeffs(sp, *T)
        mp = c.mu_p
        B = (2 * mp - c.dt) / (2 * mp + c.dt)
        A = (2 * mp - c.Pr * c.dt) / (2 * mp + c.Pr * c.dt)
        assert c.alpha ** 3 == pytest.approx(A, rel=1e-14)
        assert c.alpha ** 2 + c.nu_ref * (1 - c.alpha ** 2) == pytest.approx(B, rel=1e-13)


def test_equilibrium_is_fixed_point():
    """At T_tr = T_rot = T_vib every exchange term vanishes: the relaxation
    temperatures equal T and the targets equal the current energies."""
    sp = _sp()
    T = 3000.0
    c = _coeffs(sp, T, T, T)
    R = O.R(sp)
    ttr, trot, evr, fl = O.relaxation_temperatures(sp, c, c.alpha, T, T, T)
    assert fl == 0
    assert ttr == pytest.approx(T, rel=1e-14) and trot == pytest.approx(T, rel=1e-14)
    assert evr == pytest.approx(O.e_vib(sp, T), rel=1e-14)
    assert c.e_tr_tgt == pytest.approx(1.5 * R * T, rel=1e-14)
    assert c.e_rot_tgt == pytest.approx(R * T, rel=1e-14)
    assert c.e_vib_tgt == pytest.approx(O.e_vib(sp, T), rel=1e-14)


def test_targets_conserve_energy_and_T1_residual():
    """The three target changes sum to zero (Sec. 3.A.1), and c_v,vib(T_1) is
    the secant of e_vib between the rescaled T_tr and T_vib (App. C)."""
    sp = _sp()
    R = O.R(sp)
    for T in [(10000, 300, 300), (2000, 3000, 2500), (20000, 300, 3000), (6000, 4000, 2000)]:
        c = _coeffs(sp, *T)
        d = (c.e_tr_tgt - 1.5 * R * T[0]) + (c.e_rot_tgt - R * T[1]) + (c.e_vib_tgt - O.e_vib(sp, T[2]))
        assert abs(d) < 1e-9 * 1.5 * R * T[0]
        sec = (O.e_vib(sp, c.T_check) - O.e_vib(sp, T[2])) / (c.T_check - T[2])
        assert c.cv_T1 == pytest.approx(sec, rel=1e-12)
        # e_tr(T_check) = e_tr(T_tr) + g_tr-rot/2 (T_rot - T_tr) + g_tr-vib/2 (T_vib - T_tr)
        lhs = 1.5 * R * c.T_check
        rhs = 1.5 * R * T[0] + 0.5 * c.gamma_tr_rot * (T[1] - T[0]) + 0.5 * c.gamma_tr_vib * (T[2] - T[0])
        assert lhs == pytest.approx(rhs, rel=1e-13)
        assert c.t1_iters < 50


@pytest.mark.parametrize("delta", [1e-2, 1e-4, 1e-6])
def test_T1_iteration_near_equilibrium_stops_at_the_secant_rounding(delta):
    """Near equilibrium (T_vib just below T_tr) the secant of c_v,vib(T_1)
    cancels in its numerator; the iteration still stops within a few passes,
    and the value it returns is the secant between T_check and T_vib within
    that secant's rounding (4 eps (|e(T_check)| + |e(T_vib)|) / |T_check -
    T_vib| plus the tolerance), and within the second-order midpoint bound of
    c_v,vib at (T_check + T_vib) / 2."""
    sp = _sp()
    T = 8000.0
    for T_rot in (T, 0.9 * T):
        c = _coeffs(sp, T, T_rot, T * (1.0 - delta))
        assert c.t1_iters < 10, c.t1_iters
        ec, ev = O.e_vib(sp, c.T_check), O.e_vib(sp, T * (1.0 - delta))
        dT = c.T_check - T * (1.0 - delta)
        if abs(dT) <= 1e-9 * T:
            continue
        sec = (ec - ev) / dT
        noise = 4 * 2.0 ** -52 * (abs(ec) + abs(ev)) / abs(dT)
        assert abs(c.cv_T1 - sec) <= 2 * noise + 1e-14 * abs(sec)
        mid = O.cv_vib(sp, 0.5 * (c.T_check + T * (1.0 - delta)))
        assert c.cv_T1 == pytest.approx(mid, rel=max(1e-12, 10 * (dT / T) ** 2) + noise / mid)


def test_T1_iteration_never_cycles_near_equilibrium():
    """4,000 seeded states near equilibrium (T_vib = T_tr (1 -+ d), d log-uniform
    in [1e-9, 1e-1], T_rot within 1e-3 of T_tr): the rounded fixed-point map
    of c_v,vib(T_1) can settle into a cycle whose step exceeds the 1e-14
    relative tolerance (with that tolerance alone about 0.15 % of such states
    ran all 50 passes); stopping at the secant's rounding ends every one within
    a few passes, at the secant between T_check and T_vib within that rounding."""
    sp = _sp()
    rng = np.random.default_rng(7)
    for _ in range(4000):
        T = rng.uniform(2000.0, 20000.0)
        d = 10.0 ** rng.uniform(-9, -1) * rng.choice([-1.0, 1.0])
        Tv = T * (1.0 - d)
        c = _coeffs(sp, T, T * (1.0 + rng.normal(0.0, 1e-3)), Tv)
        assert c.t1_iters <= 6, (T, d, c.t1_iters)
        dT = c.T_check - Tv
        if abs(dT) > 1e-9 * max(abs(c.T_check), abs(Tv)):
            ec, ev = O.e_vib(sp, c.T_check), O.e_vib(sp, Tv)
            noise = 4 * 2.0 ** -52 * (abs(ec) + abs(ev)) / abs(dT)
            assert abs(c.cv_T1 - (ec - ev) / dT) <= 3 * noise + 1e-14 * abs(c.cv_T1)


def test_T1_cycle_pin_catches_the_tolerance_alone():
    """The pin above discriminates: a copy of the oracle that stops on the
    relative tolerance alone runs all 50 passes on some of the same states."""
    import ctypes as C
    src = O.source()
    old = "if (change <= 1e-14 * fabs(xn) || change <= noise) break;"
    assert old in src
    L = O.load_variant(src.replace(old, "if (change <= 1e-14 * fabs(xn)) break;"), "plant_t1_tol")
    sp = _sp()
    rng = np.random.default_rng(7)
    worst = 0
    for _ in range(4000):
        T = rng.uniform(2000.0, 20000.0)
        d = 10.0 ** rng.uniform(-9, -1) * rng.choice([-1.0, 1.0])
        Tr = T * (1.0 + rng.normal(0.0, 1e-3))
        dt = 0.5 * O.tau_c(sp, 1e23, T)
        cc = O.Coeffs()
        assert L.orc_cell_coeffs(C.byref(sp), 1e23, dt, T, Tr, T * (1.0 - d), C.byref(cc)) == 0
        worst = max(worst, cc.t1_iters)
    assert worst == 50


def _taylor_second_order(sp, c, T_tr, T_rot, T_vib, dt):
    """Second-order Taylor expansions of the energy relaxations from the
    moment production terms: Eqs. analytic_etr, and the e_rot / e_vib ones
    that follow it in Sec. 2.D."""
    R = O.R(sp)
    ctr, crot, cvib = 1.5 * R, R, O.cv_vib(sp, T_tr)
    tr, tv = c.tau_rot, c.tau_vib
    Dr = R * T_rot - R * T_tr                     # e_rot(T_rot) - e_rot(T_tr)
    Dv = O.e_vib(sp, T_vib) - O.e_vib(sp, T_tr)   # e_vib(T_vib) - e_vib(T_tr)
    etr = 1.5 * R * T_tr + (Dr / tr + Dv / tv) * dt - 0.5 * (
        (1 / tr ** 2 + crot / (ctr * tr ** 2) + cvib / (ctr * tr * tv)) * Dr
        + (1 / tv ** 2 + cvib / (ctr * tv ** 2) + crot / (ctr * tr * tv)) * Dv) * dt ** 2
    erot = R * T_rot + (-Dr / tr) * dt - 0.5 * (
        (1 / tr ** 2 + crot / (ctr * tr ** 2)) * (-Dr) + (crot / (ctr * tr * tv)) * (-Dv)) * dt ** 2
    evib = O.e_vib(sp, T_vib) + (-Dv / tv) * dt - 0.5 * (
        (1 / tv ** 2 + cvib / (ctr * tv ** 2)) * (-Dv) + (cvib / (ctr * tr * tv)) * (-Dr)) * dt ** 2
    return etr, erot, evib


@pytest.mark.parametrize("T", [(10000.0, 300.0, 300.0), (6000.0, 4000.0, 2000.0), (3000.0, 5000.0, 8000.0)])
def test_energy_targets_are_second_order(T):
    """The USP targets (Eqs. e_tr_relax..e_vib_relax) agree with the
    second-order Taylor expansion (Sec. 2.D) up to O(dt^3): halving dt divides
    the difference by ~8.  The secant c_v,vib(T_1) is what makes the
    rot-vib cross term agree at O(dt^2)."""
    sp = _sp(Z_rot=2.0, Z_vib=3.0)   # strong coupling so every term matters
    n = 1e23
    errs = []
    for f in [0.04, 0.02, 0.01]:
        dt = f * O.tau_c(sp, n, T[0])
        c = O.cell_coeffs(sp, n, dt, *T)
        ref = _taylor_second_order(sp, c, *T, dt)
        errs.append(np.array([c.e_tr_tgt - ref[0], c.e_rot_tgt - ref[1], c.e_vib_tgt - ref[2]]))
    for k in range(3):
        r1 = abs(errs[0][k] / errs[1][k])
        r2 = abs(errs[1][k] / errs[2][k])
        assert 6.5 < r1 < 9.5 and 6.5 < r2 < 9.5, (k, r1, r2)


def test_landau_teller_second_order_convergence():
    """The per-step energy recurrence of Sec. 3.A.1 converges to the
    Landau-Teller equations (Sec. 2.A) with order ~2 in dt.  omega = 1 keeps
    mu/p, hence tau_c, constant at fixed density, which is the setting of the
    Taylor analysis (App. B)."""
    sp = _sp(omega=1.0, Z_rot=5.0, Z_vib=20.0)
    R = O.R(sp)
    n = 1e23
    T0 = (10000.0, 300.0, 1000.0)
    tau_c = O.tau_c(sp, n, T0[0])
    tr, tv = 5.0 * tau_c, 20.0 * tau_c
    t_end = 40 * tau_c

    def ev_inv(e):
        return O.T_vib_from_mean_level(sp, e / (R * sp.theta_v))

    def rhs(t, y):
        etr, erot, evib = y
        Ttr, Trot, Tvib = etr / (1.5 * R), erot / R, ev_inv(evib)
        a = (R * Trot - R * Ttr) / tr
        b = (O.e_vib(sp, Tvib) - O.e_vib(sp, Ttr)) / tv
        return [a + b, -a, -b]

    y0 = [1.5 * R * T0[0], R * T0[1], O.e_vib(sp, T0[2])]
    sol = integrate.solve_ivp(rhs, (0, t_end), y0, method="DOP853", rtol=1e-12, atol=1e-6)
    ref = sol.y[:, -1]
    errs = []
    for f in [0.5, 0.25, 0.125]:
        dt = f * tau_c
        T = list(T0)
        for _ in range(int(round(t_end / dt))):
            c = O.cell_coeffs(sp, n, dt, *T)
            T = [c.e_tr_tgt / (1.5 * R), c.e_rot_tgt / R, ev_inv(c.e_vib_tgt)]
        e = np.array([1.5 * R * T[0], R * T[1], O.e_vib(sp, T[2])])
        errs.append(np.abs(e - ref).max())
    orders = [math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])]
    assert min(orders) >= 1.8, orders


# --------------------------------------------------------------------------
# samplers (Eq. update_evib) against scipy's distributions
# --------------------------------------------------------------------------
def test_nb_inversion_matches_scipy_ppf():
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(3000):
        r = int(rng.integers(1, 40))
        p = float(rng.uniform(0.2, 0.999))
        u = float(rng.uniform(0, 1))
        k, fl = O.sample_nb(r, p, u, form=0)
        assert fl == 0
        dist = stats.nbinom(r, p)
        lo = dist.cdf(k - 1) if k > 0 else 0.0
        if min(abs(u - lo), abs(u - dist.cdf(k))) < 1e-10:
            continue
        assert k == int(dist.ppf(u)), (r, p, u, k)
        checked += 1
    assert checked > 2900


def test_binomial_inversion_matches_scipy_ppf():
    rng = np.random.default_rng(12)
    for _ in range(3000):
        n = int(rng.integers(0, 60))
        p = float(rng.uniform(0.001, 0.999))
        u = float(rng.uniform(0, 1))
        k, fl = O.sample_b(n, p, u, form=0)
        assert fl == 0
        if n == 0:
            assert k == 0
            continue
        if p > 0.5:   # drawn as n - B(n, 1 - p) with the same uniform
            dist, kk = stats.binom(n, 1 - p), n - k
        else:
            dist, kk = stats.binom(n, p), k
        lo = dist.cdf(kk - 1) if kk > 0 else 0.0
        if min(abs(u - lo), abs(u - dist.cdf(kk))) < 1e-10:
            continue
        assert kk == int(dist.ppf(u)), (n, p, u, k)
    k, fl = O.sample_b(7, 1.2, 0.3, 0)
    assert k == 7 and fl & O.F_PB_CLAMP


def test_float_inversion_agrees_with_double_almost_always():
    """Form 1 decides in float; it differs from the exact inversion only when
    the uniform falls within float rounding of a cdf step."""
    rng = np.random.default_rng(13)
    diff = 0
    for _ in range(4000):
        r = int(rng.integers(1, 30)); p = float(rng.uniform(0.3, 0.99))
        u = O.uniform(int(rng.integers(0, 2 ** 32)), 1)
        diff += O.sample_nb(r, p, u, 1)[0] != O.sample_nb(r, float(np.float32(p)), u, 0)[0]
        n = int(rng.integers(0, 40)); pb = float(rng.uniform(0.01, 0.99))
        diff += O.sample_b(n, pb, u, 1)[0] != O.sample_b(n, float(np.float32(pb)), u, 0)[0]
    assert diff <= 2


def test_float_inversion_underflow_falls_back_to_double():
    # p^r underflows float for r = 200, p = 0.5; the double path must still
    # return a value near the mean r (1-p)/p = 200
    k, fl = O.sample_nb(200, 0.5, 0.5, 1)
    assert abs(k - 200) < 60 and not (fl & O.F_SAMPLER_UNDERFLOW)


def test_jump_keeps_levels_geometric():
    """Exact identity (checked here by chi^2): if I is geometric with mean e0,
    I + NB(I+1, p_NB) - B(I, p_B) is geometric with mean
    alpha^2 e0 + (1 - alpha^2) e_rel (Sec. 3.A.2 gives the mean)."""
    rng = np.random.default_rng(14)
    a2, e0, er = 0.85, 0.7, 1.6
    p_nb = 1 / (1 + er * (1 - a2))
    p_b = (1 + er) * (1 - a2)
    N = 60000
    I0 = rng.geometric(1 / (1 + e0), N) - 1
    u = rng.uniform(size=(N, 2))
    out = np.array([i + O.sample_nb(int(i) + 1, p_nb, u5, 0)[0] - O.sample_b(int(i), p_b, u6, 0)[0]
                    for i, (u5, u6) in zip(I0, u)])
    m = a2 * e0 + (1 - a2) * er
    assert out.mean() == pytest.approx(m, abs=5 * math.sqrt(m * (1 + m) / N))
    kmax = 12
    obs = np.array([(out == k).sum() for k in range(kmax)] + [(out >= kmax).sum()])
    q = m / (1 + m)
    pm = np.array([(1 - q) * q ** k for k in range(kmax)] + [q ** kmax])
    chi2 = ((obs - N * pm) ** 2 / (N * pm)).sum()
    assert stats.chi2.sf(chi2, kmax) > 1e-3


# --------------------------------------------------------------------------
# linear algebra
# --------------------------------------------------------------------------
def test_eigen_minmax_and_cholesky_against_numpy():
    rng = np.random.default_rng(15)
    for _ in range(200):
        A = rng.normal(size=(3, 3))
        S = A @ A.T + rng.uniform(-1, 1) * np.eye(3)
        P6 = [S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]]
        lo, hi = O.sym3_eig_minmax(P6)
        ev = np.linalg.eigvalsh(S)
        assert lo == pytest.approx(ev[0], abs=1e-9 * np.abs(ev).max())
        assert hi == pytest.approx(ev[-1], abs=1e-9 * np.abs(ev).max())
        ok, L6 = O.cholesky3(P6)
        assert ok == (ev[0] > 0)
        if ok:
            L = np.array([[L6[0], 0, 0], [L6[1], L6[2], 0], [L6[3], L6[4], L6[5]]])
            assert np.allclose(L @ L.T, S, rtol=1e-12, atol=1e-12 * np.abs(S).max())


# --------------------------------------------------------------------------
# one step of particles: moment relaxations of Sec. 3.A.2 in expectation
# --------------------------------------------------------------------------
def _skewed_state(rng, N, sp, T=4000.0):
    """A non-equilibrium sample with stress and all three heat fluxes."""
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
def test_one_step_stress_and_heat_flux_relaxation(form):
    """sigma^{n+1} = B sigma^n (Eq. sigma_relax) and q^{n+1} = A q^n for all
    three modes (Eqs. qtr_relax, qrot_relax, qvib_relax), in expectation,
    through a full step including the conservation scheme."""
    sp = _sp(Z_rot=5.0, Z_vib=10.0)
    rng = np.random.default_rng(16 + form)
    N = 400000
    st = _skewed_state(rng, N, sp)
    off = [0, N]
    m0 = O.moments(sp, off, st)
    n = 1e23
    dt = 0.5 * O.tau_c(sp, n, m0[4, 0])
    cc = O.cell_coeffs(sp, n, dt, m0[4, 0], m0[5, 0], m0[6, 0])
    fl, cnt = O.homog_step(sp, form, 5, 0, 1, off, [n], [dt], st)
    assert fl == 0 and cnt[O.C_CHOL_FIX] == 0
    m1 = O.moments(sp, off, st)
    s0, qt0, qr0, qv0 = _sigma_q(m0)
    s1, qt1, qr1, qv1 = _sigma_q(m1)
    R = O.R(sp)
    T = m0[4, 0]
    # statistical scale of a stress component / heat flux with N samples
    ss = R * T * math.sqrt(2.0 / N) * 4
    assert np.allclose(s1, cc.B * s0, atol=ss)
    assert np.abs(s0).max() > 20 * ss
    qs = (R * T) ** 1.5 * math.sqrt(15.0 / N) * 4
    assert np.allclose(qt1, cc.A * qt0, atol=qs)
    assert np.allclose(qr1, cc.A * qr0, atol=qs)
    qvs = (R * T) * math.sqrt(R * T) * math.sqrt(12.0 / N) * 4
    assert np.allclose(qv1, cc.A * qv0, atol=qvs)
    assert np.abs(qt0).max() > 10 * qs and np.abs(qr0).max() > 8 * qs


def test_conservation_per_cell_is_exact():
    """Sec. 4.C: momentum and total energy of each cell are conserved (FP64
    rounding only) while the modes exchange energy."""
    sp = _sp()
    w = I.batched_instances(seed=3, n_inst=6, nmin=50, nmax=3000, steps=0)
    st = O.State.from_arrays(w.particles.cx, w.particles.cy, w.particles.cz,
                             w.particles.erot, w.particles.lev)
    R = O.R(sp)
    Rth = R * sp.theta_v
    dt = np.array([0.5 * O.tau_c(sp, w.ndens[i], w.T_nominal[i, 0]) for i in range(w.n_cells)])

    def totals(s):
        out = []
        for i in range(w.n_cells):
            b, e = w.offsets[i], w.offsets[i + 1]
            mom = np.array([s.cx[b:e].sum(), s.cy[b:e].sum(), s.cz[b:e].sum()])
            en = (0.5 * (s.cx[b:e] ** 2 + s.cy[b:e] ** 2 + s.cz[b:e] ** 2) + s.erot[b:e]
                  + Rth * s.lev[b:e]).sum()
            vs = np.sqrt((s.cx[b:e] ** 2 + s.cy[b:e] ** 2 + s.cz[b:e] ** 2).sum())
            out.append((mom, en, vs))
        return out

    t0 = totals(st)
    fl, cnt = O.homog_step(sp, 0, 9, 0, 20, w.offsets, w.ndens, dt, st)
    assert fl == 0
    t1 = totals(st)
    for (m0, e0, v0), (m1, e1, _) in zip(t0, t1):
        assert np.abs(m1 - m0).max() <= 1e-12 * v0 * 10
        assert e1 == pytest.approx(e0, rel=1e-12)
    m = O.moments(sp, w.offsets, st)
    assert (m[5] > w.T_nominal[:, 1]).all()   # rotation heated by translation


def test_equilibrium_preserved():
    """At equilibrium velocities stay Maxwellian and levels geometric; the
    rotational energy keeps its mean while its second moment after one step
    is (1.5 + alpha^2 - alpha^4 / 2)(R T)^2 (from Eq. update_erot with
    exponential input), not the exponential value 2 (R T)^2."""
    sp = _sp()
    R = O.R(sp)
    T = 3000.0
    n = 1e23
    N = 300000
    rng = np.random.default_rng(17)
    p = I.equilibrium_particles(rng, N, sp.m, sp.theta_v, T_tr=T, T_rot=T, T_vib=T)
    st = O.State.from_arrays(p.cx, p.cy, p.cz, p.erot, p.lev)
    dt = 0.5 * O.tau_c(sp, n, T)
    cc = O.cell_coeffs(sp, n, dt, T, T, T)
    O.homog_step(sp, 0, 21, 0, 1, [0, N], [n], [dt], st)
    a2 = cc.alpha ** 2
    m1 = st.erot.mean()
    ratio = (st.erot ** 2).mean() / m1 ** 2
    assert ratio == pytest.approx(1.5 + a2 - a2 ** 2 / 2, abs=0.03)
    assert m1 == pytest.approx(R * T, rel=0.01)
    O.homog_step(sp, 0, 21, 1, 9, [0, N], [n], [dt], st)
    s = math.sqrt(R * T)
    for comp in (st.cx, st.cy, st.cz):
        assert stats.kstest(comp / s, "norm").pvalue > 1e-3
    q = math.exp(-sp.theta_v / T)
    kmax = 6
    obs = np.array([(st.lev == k).sum() for k in range(kmax)] + [(st.lev >= kmax).sum()])
    pm = np.array([(1 - q) * q ** k for k in range(kmax)] + [q ** kmax])
    chi2 = ((obs - N * pm) ** 2 / (N * pm)).sum()
    assert stats.chi2.sf(chi2, kmax) > 1e-4


def test_particles_follow_energy_recurrence():
    """Config-1-like relaxation: after the conservation scheme each cell energy
    equals its target (Eqs. e_rot_relax, e_vib_relax) up to the R Theta / N
    quantisation of the vibrational correction."""
    w = I.homogeneous_single(N=20000, steps=30)
    sp = O.species(**w.species)
    R = O.R(sp)
    st = O.State.from_arrays(w.particles.cx, w.particles.cy, w.particles.cz,
                             w.particles.erot, w.particles.lev)
    n = w.ndens[0]
    dt = 0.5 * O.tau_c(sp, n, w.T_nominal[0, 0])
    off = w.offsets
    Rth = R * sp.theta_v
    for s in range(30):
        m = O.moments(sp, off, st)
        cc = O.cell_coeffs(sp, n, dt, m[4, 0], m[5, 0], m[6, 0])
        etot = 1.5 * R * m[4, 0] + R * m[5, 0] + O.e_vib(sp, m[6, 0])
        fl, _ = O.homog_step(sp, 0, 1, s, 1, off, [n], [dt], st)
        assert fl == 0
        m1 = O.moments(sp, off, st)
        assert R * m1[5, 0] == pytest.approx(cc.e_rot_tgt, rel=1e-12)
        ev = O.e_vib(sp, m1[6, 0])
        assert abs(ev - cc.e_vib_tgt) <= Rth / 20000 * (1 + 1e-9)
        assert 1.5 * R * m1[4, 0] + R * m1[5, 0] + ev == pytest.approx(etot, rel=1e-12)


def test_positivity_fix_keeps_stress_relaxation():
    """Sec. 3.A.3: when D_tr is not positive definite, nu is clamped to the
    admissible range and alpha_tr re-solved from Eq. alpha_USP_positivity_1,
    which keeps alpha^2 + nu (1 - alpha^2) = B: the stress still relaxes by
    Eq. sigma_relax, in expectation, for a strongly anisotropic cell."""
    sp = _sp()
    R = O.R(sp)
    T = 4000.0
    N = 300000
    rng = np.random.default_rng(23)
    s = math.sqrt(R * T)
    g = rng.standard_normal((N, 3))
    st = O.State.from_arrays(s * math.sqrt(2.5) * g[:, 0], s * 0.5 * g[:, 1], s * 0.5 * g[:, 2],
                             rng.exponential(R * T, N),
                             (rng.geometric(1 - math.exp(-sp.theta_v / T), N) - 1).astype(np.int32))
    off = [0, N]
    n = 1e23
    m0 = O.moments(sp, off, st)
    dt = 0.5 * O.tau_c(sp, n, m0[4, 0])
    cc = O.cell_coeffs(sp, n, dt, m0[4, 0], m0[5, 0], m0[6, 0])
    fl, cnt = O.homog_step(sp, 0, 31, 0, 1, off, [n], [dt], st)
    assert cnt[O.C_CHOL_FIX] == N and not (fl & O.F_CHOL_FAIL_AFTER_FIX)
    m1 = O.moments(sp, off, st)
    s0, s1 = _sigma_q(m0)[0], _sigma_q(m1)[0]
    assert np.allclose(s1, cc.B * s0, atol=R * T * math.sqrt(8.0 / N) * 4)


def test_moments_match_brute_force_definitions():
    """Sec. 2.A moments of small cells (N <= 8) against their definitions
    evaluated term by term: U = <c>, Pi = <C C>, T_tr = tr(Pi)/3R, T_rot =
    <eps>/R, T_vib from <I>, q_tr = <C |C|^2 / 2>, q_rot = <C eps>, q_vib =
    <C I R Theta> (C = c - U); dyadic-rational states make every sum exact."""
    sp = O.species(**I.n2_vhs_relaxation_species())
    R = O.R(sp)
    rng = np.random.default_rng(17)
    sizes = [1, 2, 3, 5, 8, 8, 4]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    d = lambda: rng.integers(-64, 64, n) / 8.0
    st = O.State.from_arrays(d() * 100, d() * 100, d() * 100, np.abs(d()) * R * 50,
                             rng.integers(0, 4, n))
    m = O.moments(sp, off, st)
    for ci, N in enumerate(sizes):
        b, e = off[ci], off[ci + 1]
        c = np.stack([st.cx[b:e], st.cy[b:e], st.cz[b:e]], axis=1)
        U = sum(c[k] for k in range(N)) / N
        C = c - U
        Pi = [sum(C[k, i] * C[k, j] for k in range(N)) / N
              for i, j in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))]
        eps, lev = st.erot[b:e], st.lev[b:e]
        assert m[0, ci] == N
        assert np.array_equal(m[1:4, ci], U)
        assert np.array_equal(m[7:13, ci], Pi)
        assert m[4, ci] == pytest.approx((Pi[0] + Pi[1] + Pi[2]) / (3 * R), rel=1e-15)
        assert m[5, ci] == pytest.approx(eps.mean() / R, rel=1e-15)
        ebar = lev.mean()
        Tv = 0.0 if ebar == 0 else sp.theta_v / math.log(1.0 + 1.0 / ebar)
        assert m[6, ci] == pytest.approx(Tv, rel=1e-14)
        q = [sum(0.5 * (C[k] @ C[k]) * C[k, i] for k in range(N)) / N for i in range(3)]
        assert np.array_equal(m[13:16, ci], q)
        assert np.array_equal(m[16:19, ci], [sum(C[k, i] * eps[k] for k in range(N)) / N
                                              for i in range(3)])
        qv = [sum(C[k, i] * lev[k] for k in range(N)) / N * R * sp.theta_v for i in range(3)]
        np.testing.assert_allclose(m[19:22, ci], qv, rtol=1e-15, atol=1e-300)


@pytest.mark.parametrize("form", [0, 1])
def test_collision_draws_are_independent_normals_and_uniforms(form):
    """The four normals and two jump uniforms of a particle's step (one
    Philox block: 23-bit radius and jump uniforms, 18-bit angles; the same in
    both forms): each normal passes a KS test against N(0, 1), each uniform
    against U(0, 1), and the six are uncorrelated over 40,000 particles."""
    n = 40000
    D = np.array([np.concatenate([g, [a, b]]) for g, a, b in
                  (O.particle_draws(7, pid, 3, form) for pid in range(n))])
    for k in range(4):
        assert stats.kstest(D[:, k], "norm").pvalue > 1e-3, k
    for k in (4, 5):
        assert stats.kstest(D[:, k], "uniform").pvalue > 1e-3, k
    Z = np.column_stack([D[:, :4], stats.norm.ppf(D[:, 4:])])
    C = np.corrcoef(Z.T)
    assert np.abs(C - np.eye(6)).max() < 5.0 / math.sqrt(n)
    # float-exact uniforms, the same draws in both forms
    assert np.all(np.float32(D[:, 4]) == D[:, 4]) and np.all(np.float32(D[:, 5]) == D[:, 5])
    other = O.particle_draws(7, 123, 3, 1 - form)
    mine = O.particle_draws(7, 123, 3, form)
    assert np.array_equal(other[0], mine[0]) and other[1:] == mine[1:]
