"""ctypes binding of the plain FP64 C oracle (``usp_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.  It shares
no code with the CUDA library (``paper_2508_05642_gb300``).

Every wrapper below calls one C function of the oracle; the C source states the
passage of Kim & Jun (arXiv 2508.05642) that the function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "usp_oracle.c")
_HDR = os.path.join(_HERE, "usp_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

NMOM = 22
MOMENT_FIELDS = ["N", "Ux", "Uy", "Uz", "T_tr", "T_rot", "T_vib",
                 "Pxx", "Pyy", "Pzz", "Pxy", "Pxz", "Pyz",
                 "qtr_x", "qtr_y", "qtr_z", "qrot_x", "qrot_y", "qrot_z",
                 "qvib_x", "qvib_y", "qvib_z"]

F_PB_CLAMP = 0x01
F_CHOL_FAIL_AFTER_FIX = 0x02
F_NEG_RADICAND = 0x04
F_VIB_LOOP_CAP = 0x08
F_TREL_CLAMP = 0x10
F_SAMPLER_CAP = 0x20
F_A_NONPOS = 0x40
F_SAMPLER_UNDERFLOW = 0x80
F_WALL_CAP = 0x100
F_INFLOW_CAP = 0x800
F_CAPACITY = 0x1000

C_CHOL_FIX, C_PB_CLAMP, C_TREL_CLAMP, C_VIB_DRAWS, C_NEG_RADICAND, C_WALL_HITS, \
    C_INTERP_FALLBACK, C_SKIPPED_CELLS, C_INFLOW, C_OUTFLOW, C_NU_ZERO = range(11)
NCOUNTERS = 11


def _compile(src: str, out: str, openmp: bool) -> None:
    tmp = out + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-Wall", "-Wno-misleading-indentation",
            "-I", _HERE, src, "-o", tmp, "-lm"]
    cmd = base[:1] + (["-fopenmp"] if openmp else []) + base[1:]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and openmp:
        r = subprocess.run(base, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, out)


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liborc.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if t >= os.path.getmtime(_SRC) and t >= os.path.getmtime(_HDR):
            return _LIB_PATH
    _compile(_SRC, _LIB_PATH, openmp)
    return _LIB_PATH


def load_variant(source_text: str, tag: str):
    """Compile a modified copy of the oracle source (a test planting a
    mistake in the oracle to show that a pin catches it) into
    ``oracle/_build/liborc_<tag>.so`` and return it bound like ``lib()``.
    The regular library is not touched."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_BUILD, f"usp_oracle_{tag}.c")
    out = os.path.join(_BUILD, f"liborc_{tag}.so")
    with open(src, "w") as f:
        f.write(source_text)
    _compile(src, out, openmp=False)
    return _bind(C.CDLL(out))


def source() -> str:
    """Text of the oracle's C source."""
    with open(_SRC) as f:
        return f.read()


class Species(C.Structure):
    _fields_ = [("m", C.c_double), ("d_ref", C.c_double), ("omega", C.c_double),
                ("T_ref", C.c_double), ("c_alpha", C.c_double), ("theta_v", C.c_double),
                ("Z_rot", C.c_double), ("Z_vib", C.c_double), ("zmodel", C.c_int),
                ("Zrot_inf", C.c_double), ("T_star", C.c_double), ("C1", C.c_double),
                ("C2", C.c_double), ("sigma_vib", C.c_double)]


class Coeffs(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("n", "dt", "T_tr", "T_rot", "T_vib",
                 "mu", "p", "mu_p", "tau_c", "Z_rot", "Z_vib", "tau_rot", "tau_vib", "Pr",
                 "A", "B", "alpha", "nu_ref",
                 "g_r", "g_v", "cv_T1", "T_check", "gamma_tr_rot", "gamma_tr_vib",
                 "gamma_rot_vib")] + [("t1_iters", C.c_int)] + \
               [(n, C.c_double) for n in ("e_tr_tgt", "e_rot_tgt", "e_vib_tgt")] + \
               [("tgt_clamped", C.c_int)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class FpmCoeffs(C.Structure):
    """orc_fpm: per-cell coefficients of the plain FPM method (Sec. 2.B/2.C)."""
    _fields_ = [(n, C.c_double) for n in
                ("n", "dt", "T_tr", "T_rot", "T_vib",
                 "mu", "p", "tau_c", "Z_rot", "Z_vib", "tau_rot", "tau_vib", "Pr",
                 "nu", "tau", "alpha", "T_tr_rel", "T_rot_rel", "e_vib_rel",
                 "lam_up", "lam_dn", "e_rot_tgt", "e_vib_tgt")] + [("clamped", C.c_int)]


class Channel(C.Structure):
    _fields_ = [("ny", C.c_int), ("L", C.c_double), ("T_wall", C.c_double), ("g", C.c_double),
                ("F_num", C.c_double), ("area", C.c_double), ("reconstruct", C.c_int),
                ("method", C.c_int)]


NACC = 12
NFIELD = 13
NSURF = 180   # cylinder surface bins of the plane accumulator (ORC_NSURF)

BC_OPEN, BC_SPECULAR, BC_DIFFUSE = 0, 1, 2


class Plane(C.Structure):
    """2D plane domain (``orc_plane``): sides in the order left, right,
    bottom, top."""
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("x1", C.c_double),
                ("y0", C.c_double), ("y1", C.c_double), ("cyl_xc", C.c_double),
                ("cyl_yc", C.c_double), ("cyl_r", C.c_double), ("T_wall", C.c_double),
                ("n_inf", C.c_double), ("T_inf", C.c_double), ("U_inf", C.c_double),
                ("bc", C.c_int * 4), ("inflow", C.c_int * 4), ("F_num", C.c_double),
                ("depth", C.c_double), ("reconstruct", C.c_int), ("amr_levels", C.c_int),
                ("amr_r2", C.c_double), ("amr_r3", C.c_double), ("method", C.c_int)]


def plane(**kw) -> Plane:
    c = Plane()
    for k, v in kw.items():
        if k in ("bc", "inflow"):
            getattr(c, k)[:] = list(v)
        else:
            setattr(c, k, v)
    return c


def channel(**kw) -> Channel:
    c = Channel()
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def species(**kw) -> Species:
    s = Species()
    for k, v in kw.items():
        setattr(s, k, v)
    return s


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_U32 = C.POINTER(C.c_uint32)
_I64 = C.POINTER(C.c_int64)


def _bind(L):
    L.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
    L.orc_uniform.argtypes = [C.c_uint32, C.c_int]
    L.orc_uniform.restype = C.c_double
    for fn in ("orc_e_vib", "orc_cv_vib", "orc_T_vib_from_mean_level", "orc_mu",
               "orc_prandtl"):
        getattr(L, fn).argtypes = [C.POINTER(Species), C.c_double]
        getattr(L, fn).restype = C.c_double
    L.orc_R.argtypes = [C.POINTER(Species)]
    L.orc_R.restype = C.c_double
    L.orc_tau_c.argtypes = [C.POINTER(Species), C.c_double, C.c_double]
    L.orc_tau_c.restype = C.c_double
    L.orc_collision_numbers.argtypes = [C.POINTER(Species), C.c_double, _D, _D]
    L.orc_cell_coeffs.argtypes = [C.POINTER(Species)] + [C.c_double] * 5 + [C.POINTER(Coeffs)]
    L.orc_cell_coeffs.restype = C.c_int
    L.orc_relaxation_temperatures.argtypes = [C.POINTER(Species), C.POINTER(Coeffs), C.c_double,
                                              C.c_double, C.c_double, C.c_double, _D, _D, _D, _U32]
    L.orc_sym3_eig_minmax.argtypes = [_D, _D, _D]
    L.orc_cholesky3.argtypes = [_D, _D]
    L.orc_cholesky3.restype = C.c_int
    L.orc_sample_nb.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, _U32]
    L.orc_sample_nb.restype = C.c_int
    L.orc_sample_b.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, _U32]
    L.orc_sample_b.restype = C.c_int
    L.orc_collide_particle.argtypes = [C.POINTER(Species), C.c_int, C.POINTER(Coeffs), _D, _D,
                                       C.c_double, C.c_double, C.c_double, _D, C.c_double,
                                       C.c_double, _D, _D, _I32, _U32, _I64]
    L.orc_moments.argtypes = [C.POINTER(Species), C.c_int, _I64, _D, _D, _D, _D, _I32, _D]
    L.orc_homog_step.argtypes = [C.POINTER(Species), C.c_int, C.c_uint64, C.c_int64, C.c_int,
                                 C.c_int, _I64, _D, _D, _D, _D, _D, _D, _I32, _U32, _U32, _I64]
    L.orc_homog_step.restype = C.c_int
    L.orc_channel_step.argtypes = [C.POINTER(Species), C.c_int, C.c_uint64, C.c_int64, C.c_int,
                                   C.POINTER(Channel), C.c_double, C.c_int64, _D, _D, _D, _D, _D,
                                   _I32, _U32, _I64, _D, _U32, _I64]
    L.orc_channel_step.restype = C.c_int
    L.orc_particle_draws.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, _D, _D, _D]
    L.orc_channel_step_frozen.argtypes = L.orc_channel_step.argtypes + [C.c_void_p]
    L.orc_channel_step_frozen.restype = C.c_int
    L.orc_declog_new.restype = C.c_void_p
    L.orc_declog_free.argtypes = [C.c_void_p]
    L.orc_declog_set_mode.argtypes = [C.c_void_p, C.c_int]
    L.orc_declog_stats.argtypes = [C.c_void_p, _I64]
    L.orc_channel_reconstruct.argtypes = [C.POINTER(Channel), _I64, _D, C.c_int, C.c_double, _D]
    L.orc_wall_reemit.argtypes = [C.POINTER(Species), C.c_int, C.c_uint64, C.c_uint32,
                                  C.c_uint32, C.c_int, C.c_double, C.c_int, _D, _I32]
    L.orc_plane_step.argtypes = [C.POINTER(Species), C.c_int, C.c_uint64, C.c_int64, C.c_int,
                                 C.POINTER(Plane), _D, C.c_double, _I64, C.c_int64, _D, _D,
                                 _D, _D, _D, _D, _I32, _U32, _U32, _I64, _D, _U32, _I64]
    L.orc_plane_step.restype = C.c_int
    L.orc_plane_reconstruct.argtypes = [C.POINTER(Plane), _I64, _D, _D, C.c_int, C.c_double,
                                        C.c_double, _D]
    L.orc_inflow_flux.argtypes = [C.c_double, C.c_double, C.c_double]
    L.orc_inflow_flux.restype = C.c_double
    L.orc_inflow_normal_speed.argtypes = [C.c_double, C.c_double, C.c_uint32, C.c_uint32,
                                          C.c_uint64, C.c_int, _U32]
    L.orc_inflow_normal_speed.restype = C.c_double
    L.orc_plane_nleaf.argtypes = [C.POINTER(Plane)]
    L.orc_plane_leaves.argtypes = [C.POINTER(Plane), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.orc_plane_leaf_of.argtypes = [C.POINTER(Plane), C.c_double, C.c_double]
    L.orc_fpm_coeffs.argtypes = [C.POINTER(Species)] + [C.c_double] * 5 + \
        [C.POINTER(FpmCoeffs)]
    L.orc_gillespie.argtypes = [C.c_int, C.c_double, C.c_double, C.c_uint64, C.c_uint32,
                                C.c_uint32, C.c_int, _U32]
    L.orc_homog_step_fpm.argtypes = L.orc_homog_step.argtypes
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# ---- random numbers ---------------------------------------------------------
def philox(ctr, key) -> tuple:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return tuple(int(x) for x in out)


def particle_draws(seed, pid, step, form):
    """(G[4], u5, u6): one particle's collision draws."""
    G = np.zeros(4)
    u5, u6 = C.c_double(), C.c_double()
    lib().orc_particle_draws(C.c_uint64(seed), pid, step, form, _p(G, C.c_double),
                             C.byref(u5), C.byref(u6))
    return G, u5.value, u6.value


def uniform(x: int, form: int) -> float:
    return lib().orc_uniform(C.c_uint32(x), form)


# ---- closed forms -----------------------------------------------------------
def R(sp: Species) -> float:
    return lib().orc_R(C.byref(sp))


def e_vib(sp, T):
    return lib().orc_e_vib(C.byref(sp), T)


def cv_vib(sp, T):
    return lib().orc_cv_vib(C.byref(sp), T)


def T_vib_from_mean_level(sp, ebar):
    return lib().orc_T_vib_from_mean_level(C.byref(sp), ebar)


def mu(sp, T):
    return lib().orc_mu(C.byref(sp), T)


def tau_c(sp, n, T):
    return lib().orc_tau_c(C.byref(sp), n, T)


def prandtl(sp, T):
    return lib().orc_prandtl(C.byref(sp), T)


def collision_numbers(sp, T_tr):
    zr, zv = C.c_double(), C.c_double()
    lib().orc_collision_numbers(C.byref(sp), T_tr, C.byref(zr), C.byref(zv))
    return zr.value, zv.value


def cell_coeffs(sp, n, dt, T_tr, T_rot, T_vib) -> Coeffs:
    cc = Coeffs()
    rc = lib().orc_cell_coeffs(C.byref(sp), n, dt, T_tr, T_rot, T_vib, C.byref(cc))
    if rc != 0:
        raise ValueError("cell coefficients undefined: mu/p not positive and finite")
    return cc


def fpm_coeffs(sp, n, dt, T_tr, T_rot, T_vib) -> FpmCoeffs:
    """Per-cell coefficients of the plain FPM method."""
    fc = FpmCoeffs()
    rc = lib().orc_fpm_coeffs(C.byref(sp), n, dt, T_tr, T_rot, T_vib, C.byref(fc))
    if rc != 0:
        raise ValueError("FPM coefficients undefined: tau not positive")
    return fc


def gillespie(I, lam_up, lam_dn, seed, pid, step, form=0):
    """(new level, flags) of one particle after one step of Gillespie's method."""
    fl = C.c_uint32(0)
    k = lib().orc_gillespie(int(I), float(lam_up), float(lam_dn), C.c_uint64(seed),
                            C.c_uint32(pid), C.c_uint32(step), int(form), C.byref(fl))
    return k, fl.value


def relaxation_temperatures(sp, cc: Coeffs, alpha, T_tr, T_rot, T_vib):
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    f = C.c_uint32(0)
    lib().orc_relaxation_temperatures(C.byref(sp), C.byref(cc), alpha, T_tr, T_rot, T_vib,
                                      C.byref(a), C.byref(b), C.byref(c), C.byref(f))
    return a.value, b.value, c.value, f.value


def sym3_eig_minmax(P6):
    P = np.ascontiguousarray(P6, dtype=np.float64)
    lo, hi = C.c_double(), C.c_double()
    lib().orc_sym3_eig_minmax(_p(P, C.c_double), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def cholesky3(M6):
    M = np.ascontiguousarray(M6, dtype=np.float64)
    L = np.zeros(6)
    ok = lib().orc_cholesky3(_p(M, C.c_double), _p(L, C.c_double))
    return bool(ok), L


def sample_nb(r, p, u, form=0):
    f = C.c_uint32(0)
    k = lib().orc_sample_nb(r, p, u, form, C.byref(f))
    return k, f.value


def sample_b(n, p, u, form=0):
    f = C.c_uint32(0)
    k = lib().orc_sample_b(n, p, u, form, C.byref(f))
    return k, f.value


def collide_particle(sp, form, cc: Coeffs, U, Pi, T_tr, T_rot, T_vib, G, u5, u6, c, erot, lev):
    U = np.ascontiguousarray(U, dtype=np.float64)
    Pi = np.ascontiguousarray(Pi, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    cc_ = np.ascontiguousarray(c, dtype=np.float64).copy()
    e = C.c_double(erot)
    lv = C.c_int32(lev)
    fl = C.c_uint32(0)
    cnt = np.zeros(NCOUNTERS, dtype=np.int64)
    lib().orc_collide_particle(C.byref(sp), form, C.byref(cc), _p(U, C.c_double), _p(Pi, C.c_double),
                               T_tr, T_rot, T_vib, _p(G, C.c_double), u5, u6, _p(cc_, C.c_double),
                               C.byref(e), C.byref(lv), C.byref(fl), _p(cnt, C.c_int64))
    return cc_, e.value, lv.value, fl.value, cnt


# ---- particle-state operations ------------------------------------------------
@dataclass
class State:
    """Particle state in structure-of-arrays form, FP64 (levels int32)."""
    cx: np.ndarray
    cy: np.ndarray
    cz: np.ndarray
    erot: np.ndarray
    lev: np.ndarray
    pid: np.ndarray

    @classmethod
    def from_arrays(cls, cx, cy, cz, erot, lev, pid=None):
        n = len(cx)
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64).copy()
        if pid is None:
            pid = np.arange(n, dtype=np.uint32)
        return cls(f(cx), f(cy), f(cz), f(erot),
                   np.ascontiguousarray(lev, dtype=np.int32).copy(),
                   np.ascontiguousarray(pid, dtype=np.uint32).copy())

    def copy(self):
        return State(self.cx.copy(), self.cy.copy(), self.cz.copy(), self.erot.copy(),
                     self.lev.copy(), self.pid.copy())


def moments(sp, off, st: State) -> np.ndarray:
    off = np.ascontiguousarray(off, dtype=np.int64)
    ncell = len(off) - 1
    out = np.zeros(NMOM * ncell)
    lib().orc_moments(C.byref(sp), ncell, _p(off, C.c_int64), _p(st.cx, C.c_double),
                      _p(st.cy, C.c_double), _p(st.cz, C.c_double), _p(st.erot, C.c_double),
                      _p(st.lev, C.c_int32), _p(out, C.c_double))
    return out.reshape(NMOM, ncell)


def homog_step(sp, form, seed, step0, nsteps, off, ndens, dt, st: State):
    """Advance independent homogeneous cells ``nsteps`` steps in place.

    Returns (flags, counters)."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    ndens = np.ascontiguousarray(ndens, dtype=np.float64)
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    fl = C.c_uint32(0)
    cnt = np.zeros(NCOUNTERS, dtype=np.int64)
    rc = lib().orc_homog_step(C.byref(sp), form, C.c_uint64(seed), step0, nsteps, len(off) - 1,
                              _p(off, C.c_int64), _p(ndens, C.c_double), _p(dt, C.c_double),
                              _p(st.cx, C.c_double), _p(st.cy, C.c_double), _p(st.cz, C.c_double),
                              _p(st.erot, C.c_double), _p(st.lev, C.c_int32), _p(st.pid, C.c_uint32),
                              C.byref(fl), _p(cnt, C.c_int64))
    if rc != 0:
        raise ValueError("cell coefficients undefined in some cell (mu/p not positive and finite)")
    return fl.value, cnt


def homog_step_fpm(sp, form, seed, step0, nsteps, off, ndens, dt, st: State):
    """Advance independent homogeneous cells ``nsteps`` steps of the plain FPM
    method (Sec. 2.C) in place.

    Returns (flags, counters)."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    ndens = np.ascontiguousarray(ndens, dtype=np.float64)
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    fl = C.c_uint32(0)
    cnt = np.zeros(NCOUNTERS, dtype=np.int64)
    rc = lib().orc_homog_step_fpm(C.byref(sp), form, C.c_uint64(seed), step0, nsteps, len(off) - 1,
                              _p(off, C.c_int64), _p(ndens, C.c_double), _p(dt, C.c_double),
                              _p(st.cx, C.c_double), _p(st.cy, C.c_double), _p(st.cz, C.c_double),
                              _p(st.erot, C.c_double), _p(st.lev, C.c_int32), _p(st.pid, C.c_uint32),
                              C.byref(fl), _p(cnt, C.c_int64))
    if rc != 0:
        raise ValueError("FPM coefficients undefined in some cell")
    return fl.value, cnt


# ---- 1D channel -------------------------------------------------------------
@dataclass
class ChannelState:
    y: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    cz: np.ndarray
    erot: np.ndarray
    lev: np.ndarray
    pid: np.ndarray

    @classmethod
    def from_arrays(cls, y, cx, cy, cz, erot, lev, pid=None):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64).copy()
        n = len(y)
        if pid is None:
            pid = np.arange(n, dtype=np.uint32)
        return cls(f(y), f(cx), f(cy), f(cz), f(erot),
                   np.ascontiguousarray(lev, dtype=np.int32).copy(),
                   np.ascontiguousarray(pid, dtype=np.uint32).copy())


def channel_step(sp, form, seed, step0, nsteps, ch: Channel, dt, st: ChannelState, acc=None):
    """Advance the channel ``nsteps`` steps in place (arrays end sorted by
    cell).  Returns (cell offsets, flags, counters)."""
    n = len(st.y)
    off = np.zeros(ch.ny + 1, dtype=np.int64)
    fl = C.c_uint32(0)
    cnt = np.zeros(NCOUNTERS, dtype=np.int64)
    accp = _p(acc, C.c_double) if acc is not None else None
    rc = lib().orc_channel_step(C.byref(sp), form, C.c_uint64(seed), step0, nsteps, C.byref(ch), dt, n,
                                _p(st.y, C.c_double), _p(st.cx, C.c_double), _p(st.cy, C.c_double),
                                _p(st.cz, C.c_double), _p(st.erot, C.c_double), _p(st.lev, C.c_int32),
                                _p(st.pid, C.c_uint32), _p(off, C.c_int64), accp, C.byref(fl),
                                _p(cnt, C.c_int64))
    if rc != 0:
        raise ValueError("cell coefficients undefined in some cell (mu/p not positive and finite)")
    return off, fl.value, cnt


def channel_profiles(acc, ny: int, sp: Species):
    """Time-averaged profiles (7, ny) from the channel's pooled sums: mean
    particle count per sampled step, U (3), T_tr, T_rot, T_vib -- the sample
    means of Sec. 2.A over every particle-step of the window (T_tr from the
    pooled second moment less |U|^2, T_vib inverting e_vib at the mean
    level).  Cells that never held a particle give zeros."""
    acc = np.asarray(acc, dtype=np.float64)
    A = acc[: ny * NACC].reshape(ny, NACC)
    steps = acc[ny * NACC]
    N = A[:, 0]
    out = np.zeros((7, ny))
    m = N > 0
    Nm = N[m]
    U = A[m, 1:4] / Nm[:, None]
    Rg = R(sp)
    out[0, m] = Nm / steps if steps > 0 else 0.0
    out[1:4, m] = U.T
    out[4, m] = (A[m, 4:7].sum(axis=1) / Nm - (U ** 2).sum(axis=1)) / (3.0 * Rg)
    out[5, m] = A[m, 10] / (Nm * Rg)
    out[6, m] = [T_vib_from_mean_level(sp, e) for e in A[m, 11] / Nm]
    return out


class DecisionLog:
    """Record / replay of every discrete decision of a channel run (the
    frozen-discrete form used to check pathwise gradients by finite
    differences): ``record()`` before the base run, ``replay()`` before each
    perturbed run."""

    OFF, RECORD, REPLAY = 0, 1, 2

    def __init__(self):
        self._L = lib()
        self.h = self._L.orc_declog_new()
        if not self.h:
            raise MemoryError("orc_declog_new")

    def record(self):
        self._L.orc_declog_set_mode(self.h, self.RECORD)

    def replay(self):
        self._L.orc_declog_set_mode(self.h, self.REPLAY)

    def off(self):
        self._L.orc_declog_set_mode(self.h, self.OFF)

    def stats(self) -> dict:
        """Decisions recorded (yes/no, integer), replayed decisions that
        differ from the run's own, replay requests past the end."""
        out = np.zeros(4, dtype=np.int64)
        self._L.orc_declog_stats(self.h, _p(out, C.c_int64))
        return {"bits": int(out[0]), "ints": int(out[1]), "mismatches": int(out[2]),
                "overruns": int(out[3])}

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h:
            self._L.orc_declog_free(h)


def channel_step_frozen(sp, form, seed, step0, nsteps, ch: Channel, dt, st: ChannelState,
                        log: DecisionLog, acc=None):
    """``channel_step`` with its discrete decisions recorded into or replayed
    from ``log`` (USP-FPM method only)."""
    n = len(st.y)
    off = np.zeros(ch.ny + 1, dtype=np.int64)
    fl = C.c_uint32(0)
    cnt = np.zeros(NCOUNTERS, dtype=np.int64)
    accp = _p(acc, C.c_double) if acc is not None else None
    rc = lib().orc_channel_step_frozen(C.byref(sp), form, C.c_uint64(seed), step0, nsteps,
                                       C.byref(ch), dt, n, _p(st.y, C.c_double),
                                       _p(st.cx, C.c_double), _p(st.cy, C.c_double),
                                       _p(st.cz, C.c_double), _p(st.erot, C.c_double),
                                       _p(st.lev, C.c_int32), _p(st.pid, C.c_uint32),
                                       _p(off, C.c_int64), accp, C.byref(fl),
                                       _p(cnt, C.c_int64), C.c_void_p(log.h))
    if rc == -3:
        raise ValueError("the frozen-discrete channel step runs the USP-FPM method only")
    if rc != 0:
        raise ValueError("cell coefficients undefined in some cell (mu/p not positive and finite)")
    return off, fl.value, cnt


def channel_reconstruct(ch: Channel, counts, F, cell, y):
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(NFIELD)
    lib().orc_channel_reconstruct(C.byref(ch), _p(counts, C.c_int64), _p(F, C.c_double), cell, y,
                                  _p(out, C.c_double))
    return out


def wall_reemit(sp, form, seed, pid, step, hit, Tw, into_positive_y):
    out = np.zeros(4)
    lv = C.c_int32(0)
    lib().orc_wall_reemit(C.byref(sp), form, C.c_uint64(seed), pid, step, hit, Tw,
                          1 if into_positive_y else 0, _p(out, C.c_double), C.byref(lv))
    return out, lv.value


# ---- 2D plane (cylinder) ----------------------------------------------------
class PlaneState:
    """Particle state of the 2D plane path with spare capacity for inflow:
    the first ``n`` entries of every array are live."""

    def __init__(self, x, y, cx, cy, cz, erot, lev, cap, pid=None):
        n = len(x)
        if cap < n:
            raise ValueError("capacity below the particle count")
        self.cap = int(cap)
        self.n = n

        def f(a):
            out = np.zeros(cap)
            out[:n] = a
            return out
        self.x, self.y, self.cx, self.cy, self.cz, self.erot = map(f, (x, y, cx, cy, cz, erot))
        self.lev = np.zeros(cap, dtype=np.int32)
        self.lev[:n] = lev
        self.pid = np.zeros(cap, dtype=np.uint32)
        self.pid[:n] = np.arange(n, dtype=np.uint32) if pid is None else pid
        self.next_pid = n if pid is None else int(np.max(pid)) + 1 if n else 0

    def live(self):
        n = self.n
        return (self.x[:n], self.y[:n], self.cx[:n], self.cy[:n], self.cz[:n], self.erot[:n],
                self.lev[:n], self.pid[:n])


def plane_nleaf(pl: "Plane") -> int:
    """Number of cells (leaves) of the plane's grid, refined or not."""
    return lib().orc_plane_nleaf(C.byref(pl))


def plane_leaves(pl: "Plane"):
    """(level, ii, jj) of every leaf: level 1..3 and integer coordinates at
    its own level (centre x0 + (ii + 1/2) dx / 2^(level-1))."""
    n = plane_nleaf(pl)
    if n < 0:
        raise ValueError("refined grid: neighbouring fluid cells differ by two levels")
    lv = np.zeros(n, dtype=np.int32)
    ii = np.zeros(n, dtype=np.int32)
    jj = np.zeros(n, dtype=np.int32)
    lib().orc_plane_leaves(C.byref(pl), _p(lv, C.c_int32), _p(ii, C.c_int32), _p(jj, C.c_int32))
    return lv, ii, jj


def plane_leaf_of(pl: "Plane", x: float, y: float) -> int:
    return lib().orc_plane_leaf_of(C.byref(pl), float(x), float(y))


def plane_acc(pl: "Plane") -> np.ndarray:
    """A zeroed time-average accumulator of the plane: per-cell sums
    (NACC each), the sampled-step count, 0, then NSURF cylinder surface bins
    of 4 sums (momentum to the wall x, y; energy to the wall; events)."""
    return np.zeros(plane_nleaf(pl) * NACC + 2 + 4 * NSURF)


def plane_step(sp, form, seed, step0, nsteps, pl: Plane, area_frac, dt, st: PlaneState, acc=None):
    """Advance the plane domain ``nsteps`` steps in place (live particles end
    sorted by cell).  Returns (cell offsets, flags, counters)."""
    ncell = plane_nleaf(pl)
    if ncell < 0:
        raise ValueError("refined grid: neighbouring fluid cells differ by two levels")
    af = np.ascontiguousarray(area_frac, dtype=np.float64)
    if af.size != ncell:
        raise ValueError("area_frac needs one entry per cell")
    off = np.zeros(ncell + 1, dtype=np.int64)
    n = C.c_int64(st.n)
    npid = C.c_uint32(st.next_pid)
    fl = C.c_uint32(0)
    cnt = np.zeros(NCOUNTERS, dtype=np.int64)
    if acc is not None and acc.size < ncell * NACC + 2 + 4 * NSURF:
        raise ValueError("plane accumulator too small: use plane_acc()")
    accp = _p(acc, C.c_double) if acc is not None else None
    rc = lib().orc_plane_step(C.byref(sp), form, C.c_uint64(seed), step0, nsteps, C.byref(pl),
                              _p(af, C.c_double), dt, C.byref(n), st.cap, _p(st.x, C.c_double),
                              _p(st.y, C.c_double), _p(st.cx, C.c_double), _p(st.cy, C.c_double),
                              _p(st.cz, C.c_double), _p(st.erot, C.c_double), _p(st.lev, C.c_int32),
                              _p(st.pid, C.c_uint32), C.byref(npid), _p(off, C.c_int64), accp,
                              C.byref(fl), _p(cnt, C.c_int64))
    st.n = n.value
    st.next_pid = npid.value
    if rc != 0:
        raise ValueError("cell coefficients undefined in some cell (mu/p not positive and finite)")
    return off, fl.value, cnt


def plane_reconstruct(pl: Plane, counts, area_frac, F, cell, x, y):
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    af = np.ascontiguousarray(area_frac, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(NFIELD)
    lib().orc_plane_reconstruct(C.byref(pl), _p(counts, C.c_int64), _p(af, C.c_double),
                                _p(F, C.c_double), cell, x, y, _p(out, C.c_double))
    return out


def inflow_flux(n, RT, u_n):
    return lib().orc_inflow_flux(n, RT, u_n)


def inflow_normal_speed(RT, u_n, pid, step, seed, form=0):
    f = C.c_uint32(0)
    v = lib().orc_inflow_normal_speed(RT, u_n, pid, step, C.c_uint64(seed), form, C.byref(f))
    return v, f.value
