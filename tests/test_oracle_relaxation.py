"""Pins of the oracle's relaxation temperatures away from equilibrium.

USP-FPM (Sec. 3.A.2): the particle updates relax each mode's mean energy as
alpha^2 e(T^n) + (1 - alpha^2) e(T^rel) (the energy relaxations written
below Eqs. update_ci, update_erot and the mean-level recursion of the jump
process), and Eqs. T_tr_USP, T_rot_USP and T_vib_USP choose T^rel so that
this equals the second-order targets of Eqs. e_tr_relax, e_rot_relax and
e_vib_relax.  The targets are pinned elsewhere (energy sum, Taylor expansion,
Landau-Teller convergence); here the identity pins the relaxation
temperatures, off equilibrium where every exchange term is non-zero.

FPM (Sec. 2.B, Eqs. T_tr_FPM .. T_vib_FPM): the relaxation energies move the
three modes by exchange terms that cancel in the sum (total energy kept),
and over a small dt the FPM relaxation (1 - alpha^2)(e_rel - e) reproduces
the Landau-Teller rate of every mode, translation included.

Each pin is also run on copies of the oracle with a mistake planted in the
function it guards (a flipped sign, a misplaced 1 - alpha^2): the pin must
fail there.
"""
import ctypes as C
import math

import pytest

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I

STATES = [(10000.0, 300.0, 300.0), (2000.0, 3000.0, 2500.0), (6000.0, 4000.0, 2000.0),
          (15000.0, 1200.0, 5000.0)]
DT_OVER_TAU = [0.25, 1.0]
N_DENS = 1e23


def _sp(**over):
    d = I.n2_vhs_relaxation_species()
    d.update(over)
    return O.species(**d)


def _usp_residuals(L, sp):
    """Largest relative residual per mode of
    alpha^2 e(T^n) + (1 - alpha^2) e(T^rel) - e_target over the states."""
    R = L.orc_R(C.byref(sp))
    worst = [0.0, 0.0, 0.0]
    for T_tr, T_rot, T_vib in STATES:
        for k in DT_OVER_TAU:
            dt = k * L.orc_tau_c(C.byref(sp), N_DENS, T_tr)
            cc = O.Coeffs()
            assert L.orc_cell_coeffs(C.byref(sp), N_DENS, dt, T_tr, T_rot, T_vib, C.byref(cc)) == 0
            assert cc.tgt_clamped == 0
            ttr, trot, evr = C.c_double(), C.c_double(), C.c_double()
            fl = C.c_uint32(0)
            L.orc_relaxation_temperatures(C.byref(sp), C.byref(cc), cc.alpha, T_tr, T_rot, T_vib,
                                          C.byref(ttr), C.byref(trot), C.byref(evr), C.byref(fl))
            assert fl.value == 0
            a2 = cc.alpha ** 2
            ev = L.orc_e_vib(C.byref(sp), T_vib)
            got = [a2 * 1.5 * R * T_tr + (1 - a2) * 1.5 * R * ttr.value,
                   a2 * R * T_rot + (1 - a2) * R * trot.value,
                   a2 * ev + (1 - a2) * evr.value]
            tgt = [cc.e_tr_tgt, cc.e_rot_tgt, cc.e_vib_tgt]
            for m in range(3):
                worst[m] = max(worst[m], abs(got[m] / tgt[m] - 1.0))
    return worst


def test_usp_relaxation_temperatures_reach_the_targets():
    """Eqs. T_tr_USP / T_rot_USP / T_vib_USP against Eqs. e_tr_relax /
    e_rot_relax / e_vib_relax, to 1e-12 relative, at four non-equilibrium
    states and two time steps."""
    res = _usp_residuals(O.lib(), _sp())
    assert max(res) < 1e-12, res


def test_usp_relaxation_pin_holds_with_collision_number_models():
    """The same identity with Parker's Z_rot and Millikan-White Z_vib
    (the cylinder species), where tau_rot and tau_vib vary with T_tr."""
    d = I.cylinder_flow(nx=8, ny=4, ppc=1).species
    res = _usp_residuals(O.lib(), O.species(**d))
    assert max(res) < 1e-12, res


_USP_PLANTS = {
    # sign of the rot-vib exchange in T_rot^rel flipped
    "rotvib_sign": ("(cc->gamma_tr_rot * (T_tr - T_rot) - cc->gamma_rot_vib * (T_rot - T_vib))",
                    "(cc->gamma_tr_rot * (T_tr - T_rot) + cc->gamma_rot_vib * (T_rot - T_vib))"),
    # the tr-vib term of e_vib^rel not divided by 1 - alpha^2
    "vib_oma2": ("+ (cc->gamma_tr_vib * (T_tr - T_vib) + cc->gamma_rot_vib * (T_rot - T_vib)) / oma2;",
                 "+ cc->gamma_tr_vib * (T_tr - T_vib) + cc->gamma_rot_vib * (T_rot - T_vib) / oma2;"),
    # 3/2 R of e_tr replaced by R in T_tr^rel
    "tr_heat_capacity": ("/ (oma2 * 1.5 * R);", "/ (oma2 * R);"),
}


@pytest.mark.parametrize("name", sorted(_USP_PLANTS))
def test_usp_relaxation_pin_catches_planted_mistakes(name):
    old, new = _USP_PLANTS[name]
    src = O.source()
    assert src.count(old) == 1, "the planted edit no longer matches the oracle source"
    L = O.load_variant(src.replace(old, new), "plant_" + name)
    res = _usp_residuals(L, _sp())
    assert max(res) > 1e-6, res


def _fpm_checks(L, sp):
    """(largest relative energy-sum residual, largest relative Landau-Teller
    error of the translational mode at dt = 1e-4 tau_c)."""
    R = L.orc_R(C.byref(sp))
    sum_res, lt_err = 0.0, 0.0
    for T_tr, T_rot, T_vib in STATES:
        ev = lambda T: L.orc_e_vib(C.byref(sp), T)  # noqa: E731
        e = 1.5 * R * T_tr + R * T_rot + ev(T_vib)
        tau_c = L.orc_tau_c(C.byref(sp), N_DENS, T_tr)
        for k in (0.5, 1e-4):
            fc = O.FpmCoeffs()
            assert L.orc_fpm_coeffs(C.byref(sp), N_DENS, k * tau_c, T_tr, T_rot, T_vib,
                                    C.byref(fc)) == 0
            assert fc.clamped == 0
            e_rel = 1.5 * R * fc.T_tr_rel + R * fc.T_rot_rel + fc.e_vib_rel
            sum_res = max(sum_res, abs(e_rel / e - 1.0))
            if k == 1e-4:
                # Landau-Teller (Sec. 2.A): the translational mode gives what
                # the rotational and vibrational modes take
                zr, zv = C.c_double(), C.c_double()
                L.orc_collision_numbers(C.byref(sp), T_tr, C.byref(zr), C.byref(zv))
                rate = -((R * T_tr - R * T_rot) / (zr.value * tau_c)
                         + (ev(T_tr) - ev(T_vib)) / (zv.value * tau_c))
                a2 = fc.alpha ** 2
                de = (1 - a2) * (1.5 * R * fc.T_tr_rel - 1.5 * R * T_tr)
                lt_err = max(lt_err, abs(de / (rate * fc.dt) - 1.0))
    return sum_res, lt_err


def test_fpm_relaxation_energies_keep_energy_and_follow_landau_teller():
    """Eqs. T_tr_FPM .. T_vib_FPM: the relaxation energies sum to the
    current energy (1e-12), and the translational relaxation over a small dt
    equals minus the Landau-Teller rates of the two internal modes (first
    order in dt: within 1e-3 at dt = 1e-4 tau_c)."""
    s, lt = _fpm_checks(O.lib(), _sp(Z_rot=5.0, Z_vib=20.0))
    assert s < 1e-12 and lt < 1e-3, (s, lt)


_FPM_PLANTS = {
    "tr_vib_sign": ("+ gvib * (e_vib - orc_e_vib(sp, T_tr));",
                    "- gvib * (e_vib - orc_e_vib(sp, T_tr));"),
    "tr_rot_factor": ("double e_tr_rel = e_tr + grot * (R * T_rot - R * T_tr)",
                      "double e_tr_rel = e_tr + 2.0 * grot * (R * T_rot - R * T_tr)"),
}


@pytest.mark.parametrize("name", sorted(_FPM_PLANTS))
def test_fpm_relaxation_pin_catches_planted_mistakes(name):
    old, new = _FPM_PLANTS[name]
    src = O.source()
    assert src.count(old) == 1, "the planted edit no longer matches the oracle source"
    L = O.load_variant(src.replace(old, new), "plant_fpm_" + name)
    s, lt = _fpm_checks(L, _sp(Z_rot=5.0, Z_vib=20.0))
    assert s > 1e-6 or lt > 1e-2, (s, lt)


def test_usp_collision_moves_mean_energies_to_the_targets():
    """One collision of many particles of one cell (oracle particle update,
    cell values at every particle, no conservation step): the sample means of
    the rotational energy and level after the update equal the targets within
    five standard errors.  Off equilibrium at a time step where the exchange
    terms are several per cent of the mode energies."""
    import numpy as np
    sp = _sp(Z_rot=2.0, Z_vib=5.0)
    R = O.R(sp)
    T_tr, T_rot, T_vib = 12000.0, 2500.0, 4000.0
    dt = 1.0 * O.tau_c(sp, N_DENS, T_tr)
    cc = O.cell_coeffs(sp, N_DENS, dt, T_tr, T_rot, T_vib)
    rng = np.random.default_rng(11)
    N = 200_000
    x = math.exp(-sp.theta_v / T_vib)
    lev = (rng.geometric(1 - x, N) - 1).astype(np.int32)
    erot = rng.exponential(R * T_rot, N)
    erot *= R * T_rot / erot.mean()
    G = rng.standard_normal((N, 4))
    u = rng.random((N, 2))
    U = (C.c_double * 3)(0.0, 0.0, 0.0)
    Pi = (C.c_double * 6)(R * T_tr, R * T_tr, R * T_tr, 0.0, 0.0, 0.0)
    L = O.lib()
    new_e = np.empty(N)
    new_l = np.empty(N, dtype=np.int64)
    fl = C.c_uint32(0)
    cnt = (C.c_int64 * O.NCOUNTERS)()
    for i in range(N):
        c = (C.c_double * 3)(0.0, 0.0, 0.0)
        e = C.c_double(erot[i])
        lv = C.c_int32(int(lev[i]))
        g = (C.c_double * 4)(*G[i])
        L.orc_collide_particle(C.byref(sp), 0, C.byref(cc), U, Pi, T_tr, T_rot, T_vib, g,
                               u[i, 0], u[i, 1], c, C.byref(e), C.byref(lv), C.byref(fl), cnt)
        new_e[i] = e.value
        new_l[i] = lv.value
    assert fl.value & ~O.F_PB_CLAMP == 0
    # the exchange terms are resolvable at this sample size
    assert abs(cc.e_rot_tgt - R * T_rot) > 20 * new_e.std() / math.sqrt(N)
    assert abs(new_e.mean() - cc.e_rot_tgt) < 5 * new_e.std() / math.sqrt(N)
    # levels: E[I'] = alpha^2 <I> + (1 - alpha^2) ebar_rel, and the
    # identity above makes (1 - alpha^2) ebar_rel R Theta the vibrational
    # target less alpha^2 e_vib(T_vib)
    a2 = cc.alpha ** 2
    expect = a2 * lev.mean() + (cc.e_vib_tgt - a2 * O.e_vib(sp, T_vib)) / (R * sp.theta_v)
    assert abs(cc.e_vib_tgt - O.e_vib(sp, T_vib)) / (R * sp.theta_v) > 20 * new_l.std() / math.sqrt(N)
    assert abs(new_l.mean() - expect) < 5 * new_l.std() / math.sqrt(N)
