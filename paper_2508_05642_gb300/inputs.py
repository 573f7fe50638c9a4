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


def batched_instances(seed: int = 1, n_inst: int = 4096, nmin: float = 1e3, nmax: float = 2e5,
                      n: float = 1e23, Ttr_range=(2000.0, 20000.0), Tint_range=(300.0, 3000.0),
                      Z_rot: float = 5.0, Z_vib: float = 50.0, dt_over_tau_c: float = 0.5,
                      steps: int = 500, scale: float = 1.0) -> Workload:
    """``n_inst`` independent single-cell instances.  ``scale`` < 1 shrinks
    every particle count (for quick tests) while keeping the log-uniform mix."""
    sp = n2_vhs_relaxation_species(Z_rot, Z_vib)
    rng = np.random.default_rng([seed, 0xBA7C])
    counts = np.floor(np.exp(rng.uniform(np.log(nmin), np.log(nmax), n_inst)) * scale).astype(np.int64)
    counts = np.maximum(counts, 2)
    Ttr = rng.uniform(*Ttr_range, n_inst)
    Trot = rng.uniform(*Tint_range, n_inst)
    Tvib = rng.uniform(*Tint_range, n_inst)
    off = np.zeros(n_inst + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    Ntot = int(off[-1])
    cx = np.empty(Ntot); cy = np.empty(Ntot); cz = np.empty(Ntot)
    er = np.empty(Ntot); lev = np.empty(Ntot, dtype=np.int32)
    for i in range(n_inst):
        b, e = off[i], off[i + 1]
        p = equilibrium_particles(rng, int(e - b), sp["m"], sp["theta_v"],
                                  T_tr=Ttr[i], T_rot=Trot[i], T_vib=Tvib[i])
        cx[b:e] = p.cx; cy[b:e] = p.cy; cz[b:e] = p.cz; er[b:e] = p.erot; lev[b:e] = p.lev
    return Workload("batched homogeneous N2 relaxation, %d instances, N log-uniform [%d, %d]"
                    % (n_inst, int(nmin * scale), int(nmax * scale)), sp, off,
                    np.full(n_inst, n), np.stack([Ttr, Trot, Tvib], axis=1), dt_over_tau_c,
                    Particles(cx, cy, cz, er, lev), seed, steps)


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
