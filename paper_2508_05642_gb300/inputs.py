"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds physical constants, the workload recipes and equilibrium
(Maxwell / Boltzmann) particle sampling.  It holds none of the USP-FPM method's
arithmetic: no transport coefficient, no relaxation, no update rule.  Time steps
are given as a multiple of the mean collision time at a stated nominal state;
each side (CUDA library, oracle) evaluates that collision time itself.

Workloads (the paper's experiments are replaced by these synthetic stand-ins,
with the shapes and value ranges of Sec. 5.A):

* ``homogeneous_single``: one cell of N2, 20,000 particles, n = 1e23 m^-3,
  T_tr = 10,000 K, T_rot = T_vib = 300 K, VHS parameters d_ref = 4.17e-10 m,
  omega = 0.74, T_ref = 273 K, Z_rot = 5, Z_vib = 50, dt = 0.5 tau_c.
* ``batched_instances``: 4096 independent cells, particle counts log-uniform in
  [1e3, 2e5], T_tr ~ U[2000, 20000] K, T_rot, T_vib ~ U[300, 3000] K, same gas
  and density, dt_i = 0.5 tau_c(n, T_tr,i).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import math

import numpy as np

KB = 1.380649e-23            # Boltzmann constant [J/K]
N2_MASS = 4.65e-26           # kg; reproduces the paper's printed tau_c values
N2_THETA_V = 3371.0          # K, Sec. 5


def n2_vhs_relaxation_species(Z_rot: float = 5.0, Z_vib: float = 50.0) -> dict:
    """N2 with VHS parameters of the homogeneous relaxation workloads."""
    return dict(m=N2_MASS, d_ref=4.17e-10, omega=0.74, T_ref=273.0, c_alpha=1.0,
                theta_v=N2_THETA_V, Z_rot=Z_rot, Z_vib=Z_vib, zmodel=0,
                Zrot_inf=0.0, T_star=0.0, C1=0.0, C2=0.0, sigma_vib=0.0)


def n2_vss_species(Z_rot: float = 10.0, Z_vib: float = 50.0) -> dict:
    """N2 with the VSS parameters of the paper's table of molecular parameters."""
    return dict(m=N2_MASS, d_ref=4.11e-10, omega=0.74, T_ref=273.15, c_alpha=1.36,
                theta_v=N2_THETA_V, Z_rot=Z_rot, Z_vib=Z_vib, zmodel=0,
                Zrot_inf=0.0, T_star=0.0, C1=0.0, C2=0.0, sigma_vib=0.0)


@dataclass
class Particles:
    """Structure-of-arrays particle state (FP64 velocities/energies, int32 levels)."""
    cx: np.ndarray
    cy: np.ndarray
    cz: np.ndarray
    erot: np.ndarray
    lev: np.ndarray

    @property
    def n(self) -> int:
        return len(self.cx)

    def astype_f32_exact(self) -> "Particles":
        """Round the continuous fields to float32 and back (FP32-form inputs)."""
        r = lambda a: a.astype(np.float32).astype(np.float64)
        return Particles(r(self.cx), r(self.cy), r(self.cz), r(self.erot), self.lev.copy())


def equilibrium_particles(rng: np.random.Generator, N: int, m: float, theta_v: float,
                          U=(0.0, 0.0, 0.0), T_tr=300.0, T_rot=300.0, T_vib=300.0) -> Particles:
    """Maxwellian velocities at T_tr, exponential (two-DOF Boltzmann) specific
    rotational energies with mean R T_rot, geometric (harmonic-oscillator
    Boltzmann) vibrational levels at T_vib."""
    R = KB / m
    s = np.sqrt(R * T_tr)
    cx = U[0] + s * rng.standard_normal(N)
    cy = U[1] + s * rng.standard_normal(N)
    cz = U[2] + s * rng.standard_normal(N)
    erot = rng.exponential(R * T_rot, N) if T_rot > 0 else np.zeros(N)
    if T_vib > 0:
        x = np.exp(-theta_v / T_vib)
        lev = (rng.geometric(1.0 - x, N) - 1).astype(np.int32)
    else:
        lev = np.zeros(N, dtype=np.int32)
    return Particles(cx, cy, cz, erot, lev)


def grad17_particles(rng: np.random.Generator, N: int, m: float, theta_v: float, T_eq: float,
                     sigma_frac: float = 0.1, q_frac: float = 0.1) -> Particles:
    """N particles from Grad's 17-moment distribution at T_eq (the initial state
    of the homogeneous stress / heat-flux relaxation, Sec. 5.A.1): the
    equilibrium distribution (Maxwellian velocities, exponential rotational
    energy, geometric levels) times
      1 + sigma_ij (C_i C_j - C^2 delta_ij / 3) / (2 p R T)
        + q_tr,i C_i (C^2 - 5 R T) / (5 p (R T)^2)
        + q_rot,i C_i (eps_rot - R T) / (p (R T)^2)
        + q_vib,i C_i (sinh(x/2)/(x/2))^2 (eps_vib - e_vib(T)) / (p (R T)^2),
    x = Theta/T, p = rho R T.  Reading of the printed sigma_ij(0) = 0.1 rho R T
    (a viscous stress is traceless): the three off-diagonal components are
    sigma_frac rho R T and the diagonal ones 0; every component of the three
    heat fluxes is q_frac rho (R T)^1.5.  Sampled by acceptance from the
    equilibrium distribution with probability w / max(w) over each batch, the
    weight w clamped at 0 in the far tails (so the moments come out within a
    fraction of a per cent of the targets; the measured initial values are the
    reference of the relaxation)."""
    R = KB / m
    RT = R * T_eq
    s = math.sqrt(RT)
    x = theta_v / T_eq
    qv = math.exp(-x)
    ev_eq = R * theta_v * qv / (1.0 - qv)
    sh2 = (math.sinh(0.5 * x) / (0.5 * x)) ** 2
    sig = sigma_frac * RT          # per unit mass, off-diagonal
    qh = q_frac * RT ** 1.5        # per unit mass, every component
    out = []
    got = 0
    while got < N:
        B = max(4096, int(1.4 * (N - got)))
        c = s * rng.standard_normal((B, 3))
        er = rng.exponential(RT, B)
        lev = (rng.geometric(1.0 - qv, B) - 1).astype(np.int32)
        ev = R * theta_v * lev
        C2 = (c * c).sum(axis=1)
        csum = c.sum(axis=1)
        w = (1.0
             + sig / (RT * RT) * (c[:, 0] * c[:, 1] + c[:, 0] * c[:, 2] + c[:, 1] * c[:, 2])
             + qh / (5.0 * RT ** 3) * csum * (C2 - 5.0 * RT)
             + qh / RT ** 3 * csum * (er - RT)
             + qh / RT ** 3 * csum * sh2 * (ev - ev_eq))
        w = np.maximum(w, 0.0)
        acc = rng.uniform(0.0, w.max(), B) < w
        take = np.flatnonzero(acc)[:N - got]
        out.append((c[take], er[take], lev[take]))
        got += len(take)
    c = np.concatenate([o[0] for o in out])
    er = np.concatenate([o[1] for o in out])
    lev = np.concatenate([o[2] for o in out])
    return Particles(c[:, 0].copy(), c[:, 1].copy(), c[:, 2].copy(), er, lev)


def stress_heat_flux_relaxation(seed: int = 1, N: int = 10_000_000, dt_over_tau_c: float = 0.5,
                                t_end_over_tau_c: float = 8.0) -> Workload:
    """The homogeneous relaxation of viscous stress and heat flux of Sec. 5.A.1:
    one cell of N2 (VSS), n = 1e24 m^-3, T_tr = T_rot = T_vib = 4000 K,
    Z_rot = 10, Z_vib = 50, Grad-17 initial state with sigma(0) = 0.1 rho R T
    and q(0) = 0.1 rho (R T)^1.5, 1e7 particles; steps to t_end."""
    sp = n2_vss_species(Z_rot=10.0, Z_vib=50.0)
    rng = np.random.default_rng([seed, 0x6A17])
    T = 4000.0
    p = grad17_particles(rng, N, sp["m"], sp["theta_v"], T)
    steps = int(round(t_end_over_tau_c / dt_over_tau_c))
    return Workload("homogeneous stress / heat-flux relaxation, 1 cell x %d particles, Grad-17"
                    % N, sp, np.array([0, N], dtype=np.int64), np.array([1e24]),
                    np.array([[T, T, T]]), dt_over_tau_c, p, seed, steps)


@dataclass
class Workload:
    name: str
    species: dict
    offsets: np.ndarray          # int64, n_cells + 1
    ndens: np.ndarray            # number density per cell [1/m^3]
    T_nominal: np.ndarray        # (n_cells, 3): nominal T_tr, T_rot, T_vib
    dt_over_tau_c: float         # dt_i = factor * tau_c(ndens_i, T_tr nominal_i)
    particles: Particles
    seed: int                    # key of the method's Philox stream
    steps: int
    extra: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_particles(self) -> int:
        return int(self.offsets[-1])


def homogeneous_single(seed: int = 1, N: int = 20000, n: float = 1e23,
                       T_tr: float = 10000.0, T_rot: float = 300.0, T_vib: float = 300.0,
                       Z_rot: float = 5.0, Z_vib: float = 50.0, dt_over_tau_c: float = 0.5,
                       steps: int = 200) -> Workload:
    sp = n2_vhs_relaxation_species(Z_rot, Z_vib)
    rng = np.random.default_rng([seed, 0x5EED])
    p = equilibrium_particles(rng, N, sp["m"], sp["theta_v"], T_tr=T_tr, T_rot=T_rot, T_vib=T_vib)
    return Workload("homogeneous N2 relaxation, 1 cell x %d particles" % N, sp,
                    np.array([0, N], dtype=np.int64), np.array([n]),
                    np.array([[T_tr, T_rot, T_vib]]), dt_over_tau_c, p, seed, steps)


def batched_parameters(seed: int = 1, n_inst: int = 4096, nmin: float = 1e3, nmax: float = 2e5,
                       Ttr_range=(2000.0, 20000.0), Tint_range=(300.0, 3000.0),
                       scale: float = 1.0):
    """Per-instance particle counts (log-uniform in [nmin, nmax], times
    ``scale``, at least 2) and initial temperatures (n_inst, 3) of the batched
    workload, drawn before any particle."""
    rng = np.random.default_rng([seed, 0xBA7C])
    counts = np.floor(np.exp(rng.uniform(np.log(nmin), np.log(nmax), n_inst)) * scale).astype(np.int64)
    counts = np.maximum(counts, 2)
    Ttr = rng.uniform(*Ttr_range, n_inst)
    Trot = rng.uniform(*Tint_range, n_inst)
    Tvib = rng.uniform(*Tint_range, n_inst)
    return counts, np.stack([Ttr, Trot, Tvib], axis=1)


def batched_instances(seed: int = 1, n_inst: int = 4096, nmin: float = 1e3, nmax: float = 2e5,
                      n: float = 1e23, Ttr_range=(2000.0, 20000.0), Tint_range=(300.0, 3000.0),
                      Z_rot: float = 5.0, Z_vib: float = 50.0, dt_over_tau_c: float = 0.5,
                      steps: int = 500, scale: float = 1.0, select=None) -> Workload:
    """``n_inst`` independent single-cell instances.  ``scale`` < 1 shrinks
    every particle count (for quick tests) while keeping the log-uniform mix.
    ``select`` (instance indices, ascending) builds only those instances of
    the same population: each instance's particles come from a stream of its
    own, so a subset equals the corresponding part of the whole."""
    sp = n2_vhs_relaxation_species(Z_rot, Z_vib)
    all_counts, all_T = batched_parameters(seed, n_inst, nmin, nmax, Ttr_range, Tint_range, scale)
    idx = np.arange(n_inst) if select is None else np.asarray(select, dtype=np.int64)
    counts, T = all_counts[idx], all_T[idx]
    k = len(idx)
    off = np.zeros(k + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    Ntot = int(off[-1])
    cx = np.empty(Ntot); cy = np.empty(Ntot); cz = np.empty(Ntot)
    er = np.empty(Ntot); lev = np.empty(Ntot, dtype=np.int32)
    for j, i in enumerate(idx):
        b, e = off[j], off[j + 1]
        rng = np.random.default_rng([seed, 0xBA7C, int(i)])
        p = equilibrium_particles(rng, int(e - b), sp["m"], sp["theta_v"],
                                  T_tr=T[j, 0], T_rot=T[j, 1], T_vib=T[j, 2])
        cx[b:e] = p.cx; cy[b:e] = p.cy; cz[b:e] = p.cz; er[b:e] = p.erot; lev[b:e] = p.lev
    name = "batched homogeneous N2 relaxation, %d instances, N log-uniform [%d, %d]" % (
        n_inst, int(nmin * scale), int(nmax * scale))
    if select is not None:
        name += " (%d of them)" % k
    return Workload(name, sp, off, np.full(k, n), T, dt_over_tau_c,
                    Particles(cx, cy, cz, er, lev), seed, steps, {"instances": idx})


@dataclass
class ChannelWorkload:
    name: str
    species: dict
    channel: dict                # ny, L, T_wall, g, F_num, area, reconstruct
    dt_over_tau_c: float         # dt = factor * tau_c(n, T_wall)
    n: float                     # initial number density [1/m^3]
    y: np.ndarray
    particles: Particles
    seed: int
    steps: int
    average_last: int

    @property
    def n_particles(self) -> int:
        return len(self.y)


def channel_poiseuille(seed: int = 1, ny: int = 64, ppc: int = 200, n: float = 1.3240e23,
                       L: float = 1e-4, T_wall: float = 300.0, g: float = 5.827e7,
                       dt_over_tau_c: float = 0.2, Z_rot: float = 5.0, Z_vib: float = 50.0,
                       steps: int = 20000, average_last: int = 10000,
                       reconstruct: int = 1) -> ChannelWorkload:
    """Force-driven Poiseuille flow of N2 between diffuse plates (the set-up of
    Sec. 5.B with a body force in place of the pressure gradient): VSS N2,
    plate gap 1e-4 m (Kn = 0.1 at n = 1.324e23 m^-3), 64 cells, 200 particles
    per cell, walls at 300 K, body force 5.827e7 m/s^2 (Mach ~0.1 centreline),
    dt = 0.2 tau_c.  Particles start uniform in y at rest and equilibrium."""
    sp = n2_vss_species(Z_rot, Z_vib)
    rng = np.random.default_rng([seed, 0xC4A7])
    N = ny * ppc
    y = rng.uniform(0.0, L, N)
    p = equilibrium_particles(rng, N, sp["m"], sp["theta_v"], T_tr=T_wall, T_rot=T_wall,
                              T_vib=T_wall)
    area = 1.0
    ch = dict(ny=ny, L=L, T_wall=T_wall, g=g, F_num=n * L * area / N, area=area,
              reconstruct=reconstruct)
    return ChannelWorkload("force-driven Poiseuille N2, %d cells x %d particles" % (ny, ppc), sp,
                           ch, dt_over_tau_c, n, y, p, seed, steps, average_last)


def n2_vhs_cylinder_species() -> dict:
    """N2 with the VHS parameters of the paper's cylinder case (T_ref = 290 K,
    d_ref = 4.11e-10 m, omega = 0.70, c_alpha = 1), Parker Z_rot (Z_inf = 23,
    T* = 91.5 K) and Millikan-White with the high-temperature correction for
    Z_vib (C1 = 9.1, C2 = 220, sigma_vib = 5.81e-21 m^2), Sec. 5.C."""
    return dict(m=N2_MASS, d_ref=4.11e-10, omega=0.70, T_ref=290.0, c_alpha=1.0,
                theta_v=N2_THETA_V, Z_rot=0.0, Z_vib=0.0, zmodel=1,
                Zrot_inf=23.0, T_star=91.5, C1=9.1, C2=220.0, sigma_vib=5.81e-21)


BC_OPEN, BC_SPECULAR, BC_DIFFUSE = 0, 1, 2


def cut_cell_fractions(nx: int, ny: int, x0: float, x1: float, y0: float, y1: float,
                       xc: float, yc: float, r: float, sub: int = 64) -> np.ndarray:
    """Fluid area fraction of every cell of a uniform grid outside a circle:
    1 for cells clear of it, 0 for cells inside it, and for cells the circle
    cuts the fraction of ``sub`` x ``sub`` sub-cell midpoints outside it.
    Cell (i, j) is entry j * nx + i."""
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    i = np.arange(nx)
    j = np.arange(ny)
    xl = x0 + i * dx
    yl = y0 + j * dy
    # nearest and farthest points of each cell from the centre
    nxd = np.maximum(np.maximum(xl - xc, xc - (xl + dx)), 0.0)
    nyd = np.maximum(np.maximum(yl - yc, yc - (yl + dy)), 0.0)
    fxd = np.maximum(np.abs(xl - xc), np.abs(xl + dx - xc))
    fyd = np.maximum(np.abs(yl - yc), np.abs(yl + dy - yc))
    near2 = nyd[:, None] ** 2 + nxd[None, :] ** 2
    far2 = fyd[:, None] ** 2 + fxd[None, :] ** 2
    frac = np.ones((ny, nx))
    frac[far2 <= r * r] = 0.0
    cut = (near2 < r * r) & (far2 > r * r)
    s = (np.arange(sub) + 0.5) / sub
    for jj, ii in zip(*np.nonzero(cut)):
        px = xl[ii] + s * dx
        py = yl[jj] + s * dy
        d2 = (px[None, :] - xc) ** 2 + (py[:, None] - yc) ** 2
        frac[jj, ii] = np.count_nonzero(d2 > r * r) / float(sub * sub)
    return frac.ravel()


def refined_leaves(nx: int, ny: int, x0: float, x1: float, y0: float, y1: float,
                   xc: float, yc: float, r: float, levels: int, r2: float, r3: float):
    """Cells ("leaves") of the three-level grid of Sec. 5.C, in the order the
    plane step numbers them: level-1 cells row-major; a level-1 cell whose
    centre lies within ``r2`` of (xc, yc) is replaced by its 2 x 2 level-2
    children in the order (0,0), (1,0), (0,1), (1,1) of (x, y) halves, and
    with ``levels`` 3 a child whose centre lies within ``r3`` by its own 2 x 2
    level-3 children; a cell whose four corners lie inside the body (radius
    ``r``) is not split.  Returns (level, ii, jj) per leaf: integer
    coordinates at the leaf's own level, so that its lower-left corner is
    x0 + ii dx / 2^(level-1)."""
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny

    def within(xl, yl, w, h, rr):
        ex, ey = xl + 0.5 * w - xc, yl + 0.5 * h - yc
        return ex * ex + ey * ey < rr * rr

    def solid(xl, yl, w, h):
        if not r > 0.0:
            return False
        for q in range(4):
            ex, ey = xl + (q & 1) * w - xc, yl + (q >> 1) * h - yc
            if ex * ex + ey * ey > r * r:
                return False
        return True

    lv, li, lj = [], [], []
    for j in range(ny):
        for i in range(nx):
            xl, yl = x0 + i * dx, y0 + j * dy
            if not (levels >= 2 and within(xl, yl, dx, dy, r2) and not solid(xl, yl, dx, dy)):
                lv.append(1); li.append(i); lj.append(j)
                continue
            for k in range(4):
                xk, yk = xl + (k & 1) * 0.5 * dx, yl + (k >> 1) * 0.5 * dy
                i2, j2 = 2 * i + (k & 1), 2 * j + (k >> 1)
                if levels >= 3 and within(xk, yk, 0.5 * dx, 0.5 * dy, r3) and \
                        not solid(xk, yk, 0.5 * dx, 0.5 * dy):
                    for q in range(4):
                        lv.append(3); li.append(2 * i2 + (q & 1)); lj.append(2 * j2 + (q >> 1))
                else:
                    lv.append(2); li.append(i2); lj.append(j2)
    return (np.array(lv, dtype=np.int32), np.array(li, dtype=np.int32),
            np.array(lj, dtype=np.int32))


def refined_cut_fractions(nx: int, ny: int, x0: float, x1: float, y0: float, y1: float,
                          xc: float, yc: float, r: float, leaves) -> np.ndarray:
    """Fluid area fraction of every leaf of a refined grid (cut_cell_fractions
    on the grid of the leaf's level)."""
    lv, li, lj = leaves
    af = np.ones(len(lv))
    for L in np.unique(lv):
        k = np.nonzero(lv == L)[0]
        s = 1 << (int(L) - 1)
        if r > 0:
            fr = cut_cell_fractions(nx * s, ny * s, x0, x1, y0, y1, xc, yc, r)
            af[k] = fr[lj[k].astype(np.int64) * (nx * s) + li[k]]
    return af


@dataclass
class PlaneWorkload:
    name: str
    species: dict
    plane: dict                  # nx, ny, x0, x1, y0, y1, cyl_*, T_wall, n_inf, T_inf, U_inf,
                                 # bc[4], inflow[4], F_num, depth, reconstruct
    area_frac: np.ndarray        # fluid fraction per cell, j * nx + i
    dt_over_tau_c: float         # dt = factor * tau_c(n_inf, T_inf)
    x: np.ndarray
    y: np.ndarray
    particles: Particles
    capacity: int
    seed: int
    steps: int

    @property
    def n_particles(self) -> int:
        return len(self.x)


def cylinder_flow(seed: int = 1, nx: int = 600, ny: int = 400, ppc: float = 30.0,
                  x0: float = -0.35, x1: float = 0.40, y0: float = 0.0, y1: float = 0.50,
                  r: float = 0.1, T_wall: float = 500.0, n_inf: float = 1.2012e21,
                  T_inf: float = 200.0, U_inf: float = 2883.3, dt_over_tau_c: float = 0.5,
                  capacity_factor: float = 2.0, steps: int = 20000, reconstruct: int = 1,
                  cylinder: bool = True, amr_levels: int = 0, amr_r2: float = 0.0,
                  amr_r3: float = 0.0) -> PlaneWorkload:
    """Hypersonic N2 flow past a circular cylinder (the set-up of Sec. 5.C on a
    uniform Cartesian grid with cut cells): half body of radius 0.1 m centred on
    the origin, specular symmetry plane y = 0, fully diffuse wall at 500 K;
    Mach-10 freestream (200 K, 2883.3 m/s, n = 1.2012e21 m^-3) entering through
    the left and top sides, supersonic outflow on the right; 600 x 400 cells of
    1.25 mm, 30 particles per free cell, dt = 0.5 tau_c of the freestream.  The
    domain starts filled with the freestream (impulsive start).  With
    ``cylinder`` False the body is removed and the freestream also enters on
    the right (uniform-flow checks).  With ``amr_levels`` 2 or 3 the grid is
    refined about the body (refined_leaves): ``ppc`` particles per free
    level-1 cell, the same density in the finer cells (ppc / 4^(level-1))."""
    sp = n2_vhs_cylinder_species()
    rng = np.random.default_rng([seed, 0xC71D])
    if amr_levels >= 2:
        return _cylinder_refined(rng, sp, seed, nx, ny, ppc, x0, x1, y0, y1, r, T_wall, n_inf,
                                 T_inf, U_inf, dt_over_tau_c, capacity_factor, steps,
                                 reconstruct, cylinder, amr_levels, amr_r2, amr_r3)
    if cylinder:
        af = cut_cell_fractions(nx, ny, x0, x1, y0, y1, 0.0, 0.0, r)
    else:
        af = np.ones(nx * ny)
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    depth = 1.0
    F_num = n_inf * dx * dy * depth / ppc
    counts = np.floor(ppc * af + rng.uniform(size=nx * ny)).astype(np.int64)
    N = int(counts.sum())
    cell = np.repeat(np.arange(nx * ny), counts)
    ci, cj = cell % nx, cell // nx
    x = x0 + (ci + rng.uniform(size=N)) * dx
    y = y0 + (cj + rng.uniform(size=N)) * dy
    if cylinder:
        k = np.nonzero(x * x + y * y <= r * r)[0]
        while len(k):                  # redraw inside the cut cells' fluid part
            x[k] = x0 + (ci[k] + rng.uniform(size=len(k))) * dx
            y[k] = y0 + (cj[k] + rng.uniform(size=len(k))) * dy
            k = k[x[k] * x[k] + y[k] * y[k] <= r * r]
    p = equilibrium_particles(rng, N, sp["m"], sp["theta_v"], U=(U_inf, 0.0, 0.0), T_tr=T_inf,
                              T_rot=T_inf, T_vib=T_inf)
    pl = dict(nx=nx, ny=ny, x0=x0, x1=x1, y0=y0, y1=y1, cyl_xc=0.0, cyl_yc=0.0,
              cyl_r=r if cylinder else 0.0, T_wall=T_wall, n_inf=n_inf, T_inf=T_inf,
              U_inf=U_inf, bc=(BC_OPEN, BC_OPEN, BC_SPECULAR, BC_OPEN),
              inflow=(1, 0 if cylinder else 1, 0, 1), F_num=F_num, depth=depth,
              reconstruct=reconstruct, amr_levels=0, amr_r2=0.0, amr_r3=0.0)
    cap = int(capacity_factor * N) + 4096
    name = ("Mach-10 N2 past a cylinder, %dx%d cells, %.0f particles/cell" % (nx, ny, ppc)
            if cylinder else "uniform N2 stream, %dx%d cells" % (nx, ny))
    return PlaneWorkload(name, sp, pl, af, dt_over_tau_c, x, y, p, cap, seed, steps)


def _cylinder_refined(rng, sp, seed, nx, ny, ppc, x0, x1, y0, y1, r, T_wall, n_inf, T_inf, U_inf,
                      dt_over_tau_c, capacity_factor, steps, reconstruct, cylinder, levels, r2,
                      r3) -> PlaneWorkload:
    """cylinder_flow on the refined grid: per leaf floor(ppc af / 4^(level-1)
    + u) particles placed uniformly in it (redrawn inside it while in the
    body), so the density is the freestream's everywhere."""
    rb = r if cylinder else 0.0
    leaves = refined_leaves(nx, ny, x0, x1, y0, y1, 0.0, 0.0, rb, levels, r2, r3)
    lv, li, lj = leaves
    af = refined_cut_fractions(nx, ny, x0, x1, y0, y1, 0.0, 0.0, rb, leaves)
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    depth = 1.0
    F_num = n_inf * dx * dy * depth / ppc
    scale = 1.0 / (1 << (lv - 1)).astype(np.float64)
    counts = np.floor(ppc * af * scale * scale + rng.uniform(size=len(lv))).astype(np.int64)
    N = int(counts.sum())
    leaf = np.repeat(np.arange(len(lv)), counts)
    h, k = dx * scale[leaf], dy * scale[leaf]
    xl, yl = x0 + li[leaf] * h, y0 + lj[leaf] * k
    x = xl + rng.uniform(size=N) * h
    y = yl + rng.uniform(size=N) * k
    if cylinder:
        m = np.nonzero(x * x + y * y <= r * r)[0]
        while len(m):
            x[m] = xl[m] + rng.uniform(size=len(m)) * h[m]
            y[m] = yl[m] + rng.uniform(size=len(m)) * k[m]
            m = m[x[m] * x[m] + y[m] * y[m] <= r * r]
    p = equilibrium_particles(rng, N, sp["m"], sp["theta_v"], U=(U_inf, 0.0, 0.0), T_tr=T_inf,
                              T_rot=T_inf, T_vib=T_inf)
    pl = dict(nx=nx, ny=ny, x0=x0, x1=x1, y0=y0, y1=y1, cyl_xc=0.0, cyl_yc=0.0,
              cyl_r=rb, T_wall=T_wall, n_inf=n_inf, T_inf=T_inf,
              U_inf=U_inf, bc=(BC_OPEN, BC_OPEN, BC_SPECULAR, BC_OPEN),
              inflow=(1, 0 if cylinder else 1, 0, 1), F_num=F_num, depth=depth,
              reconstruct=reconstruct, amr_levels=levels, amr_r2=r2, amr_r3=r3)
    cap = int(capacity_factor * N) + 4096
    name = ("Mach-10 N2 past a cylinder, %dx%d level-1 cells refined to %d levels "
            "(%d cells), %.0f particles/level-1 cell" % (nx, ny, levels, len(lv), ppc))
    return PlaneWorkload(name, sp, pl, af, dt_over_tau_c, x, y, p, cap, seed, steps)


def cylinder_paper(seed: int = 1, ppc: float = 30.0, dt: float = 1.6e-7,
                   capacity_factor: float = 2.0, refined: bool = False) -> PlaneWorkload:
    """The cylinder case of Sec. 5.C with the paper's parameters: freestream
    n = 2.124e21 m^-3, 200 K, 2883 m/s (Mach 10), radius 0.1524 m, wall at
    500 K, 0.8 m x 0.6 m half domain, cells of the paper's coarse Level 1
    grid (1.25 mm: 640 x 480), its coarse time step 1.6e-7 s.  With
    ``refined`` the paper's three levels (Level 2 within 0.24 m of the
    centre, Level 3 within 0.155 m), else that uniform grid with cut cells.
    Readings: the domain spans x in [-0.4, 0.4], y in [0, 0.6] with the
    cylinder centred on the origin, and ``ppc`` particles per free level-1
    cell (the paper: 100)."""
    sp = n2_vhs_cylinder_species()
    n_inf, T_inf = 2.124e21, 200.0
    # mean collision time of the freestream (VHS, Eq. tau_c), to express dt
    ca, w = sp["c_alpha"], sp["omega"]
    mu_ref = (5.0 * (ca + 1.0) * (ca + 2.0) * math.sqrt(sp["m"] * KB * sp["T_ref"] / math.pi)
              / (4.0 * ca * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) * sp["d_ref"] ** 2))
    mu = mu_ref * (T_inf / sp["T_ref"]) ** w
    tau_c = ca * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) / (5.0 * (ca + 1.0) * (ca + 2.0)) \
        * mu / (n_inf * KB * T_inf)
    wl = cylinder_flow(seed=seed, nx=640, ny=480, ppc=ppc, x0=-0.4, x1=0.4, y0=0.0, y1=0.6,
                       r=0.1524, T_wall=500.0, n_inf=n_inf, T_inf=T_inf, U_inf=2883.0,
                       dt_over_tau_c=dt / tau_c, capacity_factor=capacity_factor,
                       amr_levels=3 if refined else 0, amr_r2=0.24 if refined else 0.0,
                       amr_r3=0.155 if refined else 0.0)
    wl.name = ("Mach-10 N2 past a 0.1524 m cylinder (Sec. 5.C parameters), 640x480 %s, "
               "%.0f particles/%s, dt = %.3g s"
               % ("level-1 cells on 3 levels (%d cells)" % len(wl.area_frac) if refined
                  else "cells", ppc, "level-1 cell" if refined else "cell", dt))
    return wl
