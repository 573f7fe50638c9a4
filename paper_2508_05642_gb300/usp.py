"""Thin ctypes binding of ``libusp.so`` (C ABI in ``include/usp.h``).

Argument marshalling only: every step of the particle update runs in the CUDA
kernels of the library.  The functions keep the C names.  Importing this
module never falls back to anything: if the library cannot be built or loaded
the call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

USP_OK, USP_EINVAL, USP_ENOMEM, USP_ECUDA, USP_EDEVICE, USP_ENOTSUP = 0, -1, -2, -3, -4, -5
USP_FP64, USP_FP32, USP_FP64_TANGENT, USP_FP32_TANGENT = 0, 1, 2, 3
TANGENT_FORMS = (USP_FP64_TANGENT, USP_FP32_TANGENT)
USP_NMOM = 22
USP_NCOUNTERS = 11

F_PB_CLAMP = 0x01
F_CHOL_FAIL_AFTER_FIX = 0x02
F_NEG_RADICAND = 0x04
F_VIB_LOOP_CAP = 0x08
F_TREL_CLAMP = 0x10
F_SAMPLER_CAP = 0x20
F_A_NONPOS = 0x40
F_SAMPLER_UNDERFLOW = 0x80
F_BOUNDS = 0x200
F_INFLOW_CAP = 0x800
F_CAPACITY = 0x1000
F_WAIT_TIMEOUT = 0x400
ERROR_FLAGS = F_A_NONPOS | F_SAMPLER_UNDERFLOW | F_BOUNDS | F_WAIT_TIMEOUT | F_CAPACITY

C_CHOL_FIX, C_PB_CLAMP, C_TREL_CLAMP, C_VIB_DRAWS, C_NEG_RADICAND, C_WALL_HITS, \
    C_INTERP_FALLBACK, C_SKIPPED_CELLS, C_INFLOW, C_OUTFLOW, C_NU_ZERO = range(11)

EXPORTED = ["usp_select_device", "usp_tau_c", "usp_strerror", "usp_init_homogeneous", "usp_step", "usp_moments",
            "usp_get_particles", "usp_set_particles", "usp_step_host", "usp_status", "usp_sync",
            "usp_info", "usp_tuning", "usp_set_variant", "usp_launch_count", "usp_profile_enable", "usp_profile_read",
            "usp_moments_noalloc", "usp_init_channel", "usp_channel_sample",
            "usp_channel_read", "usp_channel_get_particles", "usp_init_plane", "usp_plane_leaves", "usp_plane_count",
            "usp_plane_get_particles", "usp_sample", "usp_sample_read", "usp_profiles",
            "usp_backward", "usp_checkpoint_bytes", "usp_save", "usp_load", "usp_set_wait_limit",
            "usp_wait_check", "usp_guide_row", "usp_destroy"]
USP_METHOD_USP_FPM, USP_METHOD_FPM = 0, 1
USP_NSURF = 180
USP_NOALLOC_MAX_CELLS = 8192
USP_NPROF = 7


class usp_species(C.Structure):
    _fields_ = [("m", C.c_double), ("d_ref", C.c_double), ("omega", C.c_double),
                ("T_ref", C.c_double), ("c_alpha", C.c_double), ("theta_v", C.c_double),
                ("Z_rot", C.c_double), ("Z_vib", C.c_double), ("zmodel", C.c_int),
                ("Zrot_inf", C.c_double), ("T_star", C.c_double), ("C1", C.c_double),
                ("C2", C.c_double), ("sigma_vib", C.c_double)]


class usp_channel(C.Structure):
    _fields_ = [("ny", C.c_int), ("L", C.c_double), ("T_wall", C.c_double), ("g", C.c_double),
                ("F_num", C.c_double), ("area", C.c_double), ("reconstruct", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


USP_BC_OPEN, USP_BC_SPECULAR, USP_BC_DIFFUSE = 0, 1, 2


class usp_plane(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("x1", C.c_double),
                ("y0", C.c_double), ("y1", C.c_double), ("cyl_xc", C.c_double),
                ("cyl_yc", C.c_double), ("cyl_r", C.c_double), ("T_wall", C.c_double),
                ("n_inf", C.c_double), ("T_inf", C.c_double), ("U_inf", C.c_double),
                ("bc", C.c_int * 4), ("inflow", C.c_int * 4), ("F_num", C.c_double),
                ("depth", C.c_double), ("reconstruct", C.c_int), ("amr_levels", C.c_int),
                ("amr_r2", C.c_double), ("amr_r3", C.c_double)]


class usp_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("seed", C.c_uint64), ("step0", C.c_int64),
                ("stream", C.c_void_p), ("use_graph", C.c_int), ("tile", C.c_int),
                ("alloc", ALLOC_FN), ("free_", FREE_FN), ("alloc_user", C.c_void_p),
                ("method", C.c_int)]


_lock = threading.Lock()
_lib = None
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_U32 = C.POINTER(C.c_uint32)
_CTX = C.c_void_p


def library_path() -> str:
    return _build.LIB


def lib():
    """Build (if stale) and load libusp.so; raises if either fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            L.usp_select_device.argtypes = [C.c_int]
            L.usp_tau_c.argtypes = [C.POINTER(usp_species), C.c_double, C.c_double]
            L.usp_tau_c.restype = C.c_double
            L.usp_strerror.argtypes = [C.c_int]
            L.usp_strerror.restype = C.c_char_p
            L.usp_init_homogeneous.argtypes = [C.POINTER(_CTX), C.POINTER(usp_species),
                                               C.POINTER(usp_config), C.c_int, _I64, _D, _D,
                                               _D, _D, _D, _D, _I32]
            L.usp_step.argtypes = [_CTX, C.c_int]
            L.usp_moments.argtypes = [_CTX, C.c_void_p, C.c_int]
            L.usp_get_particles.argtypes = [_CTX, _D, _D, _D, _D, _I32]
            L.usp_set_particles.argtypes = [_CTX, _D, _D, _D, _D, _I32]
            L.usp_step_host.argtypes = [_CTX, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        _I32, C.c_int, _D, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, _I32]
            L.usp_status.argtypes = [_CTX, _U32, _I64, C.c_int]
            L.usp_sync.argtypes = [_CTX]
            L.usp_info.argtypes = [_CTX, _I64, C.POINTER(C.c_int), C.POINTER(C.c_int), _I64,
                                   C.POINTER(C.c_int), _I64]
            L.usp_tuning.argtypes = [_CTX, C.POINTER(C.c_int), C.POINTER(C.c_int), _D]
            L.usp_set_variant.argtypes = [_CTX, C.c_int, C.c_int]
            L.usp_launch_count.argtypes = [_CTX]
            L.usp_launch_count.restype = C.c_int64
            L.usp_profile_enable.argtypes = [_CTX, C.c_int]
            L.usp_profile_read.argtypes = [_CTX, _D, _I64]
            L.usp_moments_noalloc.argtypes = [C.POINTER(usp_species), C.c_int, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_void_p]
            L.usp_init_channel.argtypes = [C.POINTER(_CTX), C.POINTER(usp_species),
                                           C.POINTER(usp_config), C.POINTER(usp_channel),
                                           C.c_double, C.c_int64, _D, _D, _D, _D, _D, _I32, _U32]
            L.usp_channel_sample.argtypes = [_CTX, C.c_int]
            L.usp_channel_read.argtypes = [_CTX, _D, C.c_int]
            L.usp_channel_get_particles.argtypes = [_CTX, _D, _D, _D, _D, _D, _I32, _U32]
            L.usp_init_plane.argtypes = [C.POINTER(_CTX), C.POINTER(usp_species),
                                         C.POINTER(usp_config), C.POINTER(usp_plane), C.c_double,
                                         _D, C.c_int64, C.c_int64, _D, _D, _D, _D, _D, _D, _I32,
                                         _U32]
            L.usp_plane_count.argtypes = [_CTX, _I64, _U32]
            L.usp_plane_leaves.argtypes = [C.POINTER(usp_plane), C.POINTER(C.c_int32),
                                           C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
            L.usp_plane_get_particles.argtypes = [_CTX, C.c_int64, _I64, _D, _D, _D, _D, _D, _D,
                                                  _I32, _U32]
            L.usp_sample.argtypes = [_CTX, C.c_int]
            L.usp_sample_read.argtypes = [_CTX, _D, C.c_int]
            L.usp_profiles.argtypes = [_CTX, C.c_void_p, C.c_int]
            L.usp_backward.argtypes = [_CTX, C.c_void_p, C.c_void_p, C.c_int]
            L.usp_checkpoint_bytes.argtypes = [_CTX, C.POINTER(C.c_size_t)]
            L.usp_save.argtypes = [_CTX, C.c_void_p, C.c_int]
            L.usp_load.argtypes = [_CTX, C.c_void_p, C.c_int]
            L.usp_set_wait_limit.argtypes = [_CTX, C.c_int64]
            L.usp_wait_check.argtypes = [_CTX, C.c_int64]
            L.usp_guide_row.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
            L.usp_destroy.argtypes = [_CTX]
            L.usp_destroy.restype = None
            _lib = L
    return _lib


class USPError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {usp_strerror(code)} ({code})")
        self.code = code


def _check(rc, where):
    if rc != USP_OK:
        raise USPError(rc, where)


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def usp_strerror(code: int) -> str:
    return lib().usp_strerror(code).decode()


def make_species(d: dict) -> usp_species:
    s = usp_species()
    for k, _ in usp_species._fields_:
        setattr(s, k, d.get(k, 0))
    return s


def usp_select_device(dev: int):
    _check(lib().usp_select_device(dev), "usp_select_device")


def usp_tau_c(species: dict, n: float, T: float) -> float:
    return lib().usp_tau_c(C.byref(make_species(species)), n, T)


class Context:
    """Owns one ``usp_ctx``; methods map 1:1 onto the C entry points."""

    def __init__(self, handle, n_particles, n_cells, precision, keepalive, kind=0):
        self.h = handle
        self.n_particles = n_particles
        self.n_cells = n_cells
        self.precision = precision
        self._keep = keepalive
        self.kind = kind          # 0 homogeneous, 1 channel, 2 plane

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "h", None):
            lib().usp_destroy(self.h)
            self.h = None


def usp_init_homogeneous(species: dict, offsets, ndens, dt, cx, cy, cz, erot, lev, *,
                         precision=USP_FP32, seed=1, step0=0, stream=None, use_graph=True,
                         tile=0, allocator=None, method=0) -> Context:
    """Create a context for independent homogeneous cells; arrays are host numpy.
    ``method``: USP_METHOD_USP_FPM (0) or USP_METHOD_FPM (1)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nd = np.ascontiguousarray(ndens, dtype=np.float64)
    dtv = np.ascontiguousarray(dt, dtype=np.float64)
    f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    cx, cy, cz, erot = f(cx), f(cy), f(cz), f(erot)
    lev = np.ascontiguousarray(lev, dtype=np.int32)
    cfg = usp_config()
    cfg.precision = precision
    cfg.seed = seed
    cfg.step0 = step0
    cfg.stream = stream or None
    cfg.use_graph = 1 if use_graph else 0
    cfg.tile = tile
    cfg.method = int(method)
    keep = []
    if allocator is not None:
        a_fn, f_fn, user = allocator
        cfg.alloc = a_fn
        cfg.free_ = f_fn
        cfg.alloc_user = user
        keep += [a_fn, f_fn]
    sp = make_species(species)
    h = _CTX()
    rc = lib().usp_init_homogeneous(C.byref(h), C.byref(sp), C.byref(cfg), len(off) - 1,
                                    _p(off, C.c_int64), _p(nd, C.c_double), _p(dtv, C.c_double),
                                    _p(cx, C.c_double), _p(cy, C.c_double), _p(cz, C.c_double),
                                    _p(erot, C.c_double), _p(lev, C.c_int32))
    _check(rc, "usp_init_homogeneous")
    return Context(h, int(off[-1]), len(off) - 1, precision, keep)


def usp_init_channel(species: dict, channel: dict, dt: float, y, cx, cy, cz, erot, lev, pid=None,
                     *, precision=USP_FP32, seed=1, step0=0, stream=None, use_graph=True,
                     allocator=None, method=USP_METHOD_USP_FPM) -> Context:
    """Create a 1D-channel context (host numpy inputs)."""
    f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    y, cx, cy, cz, erot = f(y), f(cx), f(cy), f(cz), f(erot)
    lev = np.ascontiguousarray(lev, dtype=np.int32)
    pidp = None
    if pid is not None:
        pid = np.ascontiguousarray(pid, dtype=np.uint32)
        pidp = _p(pid, C.c_uint32)
    cfg = usp_config()
    cfg.precision = precision
    cfg.seed = seed
    cfg.step0 = step0
    cfg.stream = stream or None
    cfg.use_graph = 1 if use_graph else 0
    cfg.method = method
    keep = []
    if allocator is not None:
        a_fn, f_fn, user = allocator
        cfg.alloc, cfg.free_, cfg.alloc_user = a_fn, f_fn, user
        keep += [a_fn, f_fn]
    ch = usp_channel()
    for k, _ in usp_channel._fields_:
        setattr(ch, k, channel[k])
    sp = make_species(species)
    h = _CTX()
    n = len(y)
    rc = lib().usp_init_channel(C.byref(h), C.byref(sp), C.byref(cfg), C.byref(ch), dt, n,
                                _p(y, C.c_double), _p(cx, C.c_double), _p(cy, C.c_double),
                                _p(cz, C.c_double), _p(erot, C.c_double), _p(lev, C.c_int32), pidp)
    _check(rc, "usp_init_channel")
    return Context(h, n, int(channel["ny"]), precision, keep, kind=1)


def usp_channel_sample(ctx: Context, on: bool = True):
    _check(lib().usp_channel_sample(ctx.h, 1 if on else 0), "usp_channel_sample")


def usp_channel_read(ctx: Context, reset: bool = False, blocks: int = None) -> np.ndarray:
    """ny * 12 + 2 doubles: per-cell time-average sums, step count, wall
    momentum (four such blocks in the tangent forms: sums, then their
    derivatives with respect to Z_rot, omega, T_wall)."""
    if blocks is None:
        blocks = 4 if ctx.precision in TANGENT_FORMS else 1
    out = np.zeros((ctx.n_cells * 12 + 2) * blocks)
    _check(lib().usp_channel_read(ctx.h, _p(out, C.c_double), 1 if reset else 0),
           "usp_channel_read")
    return out


def usp_channel_get_particles(ctx: Context):
    n = ctx.n_particles
    y, cx, cy, cz, er = (np.zeros(n) for _ in range(5))
    lev = np.zeros(n, dtype=np.int32)
    pid = np.zeros(n, dtype=np.uint32)
    _check(lib().usp_channel_get_particles(ctx.h, *[_p(a, C.c_double) for a in (y, cx, cy, cz, er)],
                                           _p(lev, C.c_int32), _p(pid, C.c_uint32)),
           "usp_channel_get_particles")
    return y, cx, cy, cz, er, lev, pid


def make_plane(plane: dict) -> usp_plane:
    """usp_plane from a dict of its fields (refinement fields default to the
    uniform grid)."""
    pl = usp_plane()
    for k, _ in usp_plane._fields_:
        if k in ("bc", "inflow"):
            getattr(pl, k)[:] = list(plane[k])
        elif k.startswith("amr_"):
            setattr(pl, k, plane.get(k, 0))
        else:
            setattr(pl, k, plane[k])
    return pl


def usp_plane_leaves(plane: dict, arrays: bool = False):
    """Cell count of a plane's grid, or with ``arrays`` (level, ii, jj) per
    cell (usp_plane_leaves)."""
    pl = make_plane(plane)
    n = lib().usp_plane_leaves(C.byref(pl), None, None, None)
    _check(n if n < 0 else 0, "usp_plane_leaves")
    if not arrays:
        return n
    lv, ii, jj = (np.zeros(n, dtype=np.int32) for _ in range(3))
    lib().usp_plane_leaves(C.byref(pl), _p(lv, C.c_int32), _p(ii, C.c_int32), _p(jj, C.c_int32))
    return lv, ii, jj


def usp_init_plane(species: dict, plane: dict, dt: float, area_frac, x, y, cx, cy, cz, erot, lev,
                   capacity: int, pid=None, *, precision=USP_FP32, seed=1, step0=0, stream=None,
                   use_graph=True, allocator=None, method=USP_METHOD_USP_FPM) -> Context:
    """Create a 2D plane context (host numpy inputs); ``method`` USP_METHOD_FPM
    runs the plain FPM method with the cell values."""
    f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    x, y, cx, cy, cz, erot, af = f(x), f(y), f(cx), f(cy), f(cz), f(erot), f(area_frac)
    lev = np.ascontiguousarray(lev, dtype=np.int32)
    pidp = None
    if pid is not None:
        pid = np.ascontiguousarray(pid, dtype=np.uint32)
        pidp = _p(pid, C.c_uint32)
    cfg = usp_config()
    cfg.precision = precision
    cfg.seed = seed
    cfg.step0 = step0
    cfg.stream = stream or None
    cfg.use_graph = 1 if use_graph else 0
    cfg.method = method
    keep = []
    if allocator is not None:
        a_fn, f_fn, user = allocator
        cfg.alloc, cfg.free_, cfg.alloc_user = a_fn, f_fn, user
        keep += [a_fn, f_fn]
    pl = make_plane(plane)
    ncell = usp_plane_leaves(plane)
    sp = make_species(species)
    h = _CTX()
    n = len(x)
    rc = lib().usp_init_plane(C.byref(h), C.byref(sp), C.byref(cfg), C.byref(pl), dt,
                              _p(af, C.c_double), n, int(capacity), _p(x, C.c_double),
                              _p(y, C.c_double), _p(cx, C.c_double), _p(cy, C.c_double),
                              _p(cz, C.c_double), _p(erot, C.c_double), _p(lev, C.c_int32), pidp)
    _check(rc, "usp_init_plane")
    ctx = Context(h, n, ncell, precision, keep, kind=2)
    ctx.capacity = int(capacity)
    return ctx


def usp_plane_count(ctx: Context):
    """(live particle count, id of the next entering particle)."""
    n = np.zeros(1, dtype=np.int64)
    nxt = np.zeros(1, dtype=np.uint32)
    _check(lib().usp_plane_count(ctx.h, _p(n, C.c_int64), _p(nxt, C.c_uint32)), "usp_plane_count")
    return int(n[0]), int(nxt[0])


def usp_plane_get_particles(ctx: Context):
    """x, y, cx, cy, cz, erot, lev, pid of the live particles (cell order)."""
    cap = ctx.capacity
    out = [np.zeros(cap) for _ in range(6)]
    lev = np.zeros(cap, dtype=np.int32)
    pid = np.zeros(cap, dtype=np.uint32)
    n = np.zeros(1, dtype=np.int64)
    _check(lib().usp_plane_get_particles(ctx.h, cap, _p(n, C.c_int64),
                                         *[_p(a, C.c_double) for a in out], _p(lev, C.c_int32),
                                         _p(pid, C.c_uint32)), "usp_plane_get_particles")
    k = int(n[0])
    return tuple(a[:k] for a in out) + (lev[:k], pid[:k])


def usp_sample(ctx: Context, on: bool = True):
    _check(lib().usp_sample(ctx.h, 1 if on else 0), "usp_sample")


def usp_sample_read(ctx: Context, reset: bool = False) -> np.ndarray:
    """Per-cell time-average sums of a channel or plane context (n_cells * 12
    + 2 doubles; a plane context appends USP_NSURF x 4 cylinder surface sums)."""
    blocks = 4 if ctx.precision in TANGENT_FORMS else 1
    extra = 4 * USP_NSURF if ctx.kind == 2 else 0
    out = np.zeros((ctx.n_cells * 12 + 2) * blocks + extra)
    _check(lib().usp_sample_read(ctx.h, _p(out, C.c_double), 1 if reset else 0),
           "usp_sample_read")
    return out


def usp_profiles(ctx: Context, out=None, out_is_device=False):
    """Time-averaged channel profiles (USP_NPROF x ny; in the tangent
    form 4 x USP_NPROF x ny: values, then derivatives w.r.t. Z_rot, omega,
    T_wall).  Host numpy unless a device pointer (int) is given."""
    blocks = 4 if ctx.precision in TANGENT_FORMS else 1
    if out_is_device:
        _check(lib().usp_profiles(ctx.h, C.c_void_p(out), 1), "usp_profiles")
        return None
    o = np.zeros((blocks, USP_NPROF, ctx.n_cells), dtype=np.float64)
    _check(lib().usp_profiles(ctx.h, o.ctypes.data_as(C.c_void_p), 0), "usp_profiles")
    return o if blocks > 1 else o[0]


def usp_backward(ctx: Context, d_dL: int, grad3=None, grad_is_device=False):
    """Gradient (3,) of an objective w.r.t. (Z_rot, omega, T_wall) from
    dL/dprofiles held in device memory at ``d_dL`` (USP_NPROF x ny doubles).
    With grad_is_device, ``grad3`` is a device pointer written asynchronously."""
    if grad_is_device:
        _check(lib().usp_backward(ctx.h, C.c_void_p(d_dL), C.c_void_p(grad3), 1), "usp_backward")
        return None
    g = np.zeros(3)
    _check(lib().usp_backward(ctx.h, C.c_void_p(d_dL), g.ctypes.data_as(C.c_void_p), 0),
           "usp_backward")
    return g


def usp_checkpoint_bytes(ctx: Context) -> int:
    n = C.c_size_t(0)
    _check(lib().usp_checkpoint_bytes(ctx.h, C.byref(n)), "usp_checkpoint_bytes")
    return int(n.value)


def usp_save(ctx: Context, buf=None, buf_is_device=False):
    """Checkpoint into ``buf`` (a host numpy uint8 array of
    usp_checkpoint_bytes, allocated when None; or a device pointer with
    buf_is_device).  Returns the host array (or None)."""
    if buf_is_device:
        _check(lib().usp_save(ctx.h, C.c_void_p(buf), 1), "usp_save")
        return None
    if buf is None:
        buf = np.zeros(usp_checkpoint_bytes(ctx), dtype=np.uint8)
    _check(lib().usp_save(ctx.h, buf.ctypes.data_as(C.c_void_p), 0), "usp_save")
    return buf


def usp_load(ctx: Context, buf, buf_is_device=False):
    if buf_is_device:
        _check(lib().usp_load(ctx.h, C.c_void_p(buf), 1), "usp_load")
        return
    b = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().usp_load(ctx.h, b.ctypes.data_as(C.c_void_p), 0), "usp_load")


def usp_step(ctx: Context, nsteps: int):
    _check(lib().usp_step(ctx.h, nsteps), "usp_step")


def usp_moments(ctx: Context, out=None, out_is_device=False) -> np.ndarray:
    """Per-cell moments (USP_NMOM x n_cells); host numpy unless a device
    pointer (int) is given with out_is_device=True."""
    if out_is_device:
        _check(lib().usp_moments(ctx.h, C.c_void_p(out), 1), "usp_moments")
        return None
    o = np.zeros((USP_NMOM, ctx.n_cells), dtype=np.float64)
    _check(lib().usp_moments(ctx.h, o.ctypes.data_as(C.c_void_p), 0), "usp_moments")
    return o


def usp_get_particles(ctx: Context):
    n = ctx.n_particles
    out = [np.zeros(n) for _ in range(4)] + [np.zeros(n, dtype=np.int32)]
    _check(lib().usp_get_particles(ctx.h, *[_p(a, C.c_double) for a in out[:4]],
                                   _p(out[4], C.c_int32)), "usp_get_particles")
    return out


def usp_set_particles(ctx: Context, cx, cy, cz, erot, lev):
    f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    arrs = [f(cx), f(cy), f(cz), f(erot)]
    lv = np.ascontiguousarray(lev, dtype=np.int32)
    _check(lib().usp_set_particles(ctx.h, *[_p(a, C.c_double) for a in arrs],
                                   _p(lv, C.c_int32)), "usp_set_particles")


def usp_step_host(ctx: Context, cx, cy, cz, erot, lev, nsteps: int, moments_out: np.ndarray,
                  out=None):
    """End-to-end call on host buffers (ideally pinned); arrays in the
    context's precision.  ``out`` = (cx, cy, cz, erot, lev) host arrays or None."""
    ptr = lambda a: C.c_void_p(a.ctypes.data) if isinstance(a, np.ndarray) else C.c_void_p(a)
    lv = lev.ctypes.data_as(_I32) if isinstance(lev, np.ndarray) else C.cast(lev, _I32)
    o = [None] * 5 if out is None else out
    olv = None if o[4] is None else (o[4].ctypes.data_as(_I32) if isinstance(o[4], np.ndarray)
                                     else C.cast(o[4], _I32))
    rc = lib().usp_step_host(ctx.h, ptr(cx), ptr(cy), ptr(cz), ptr(erot), lv, nsteps,
                             _p(moments_out, C.c_double),
                             *(None if a is None else ptr(a) for a in o[:4]), olv)
    _check(rc, "usp_step_host")


def usp_status(ctx: Context, reset=False):
    f = C.c_uint32(0)
    cnt = np.zeros(USP_NCOUNTERS, dtype=np.int64)
    rc = lib().usp_status(ctx.h, C.byref(f), _p(cnt, C.c_int64), 1 if reset else 0)
    if rc not in (USP_OK, USP_EDEVICE):
        _check(rc, "usp_status")
    return f.value, cnt


def usp_guide_row(row, n_flip: int = -1) -> np.ndarray:
    """The 256-byte guide of one 48-value jump-table row (host code)."""
    r = np.ascontiguousarray(row, dtype=np.float32)
    if r.shape != (48,):
        raise ValueError("a jump-table row holds 48 values")
    g = np.zeros(256, dtype=np.uint8)
    _check(lib().usp_guide_row(r.ctypes.data_as(C.c_void_p), int(n_flip), g.ctypes.data_as(C.c_void_p)),
           "usp_guide_row")
    return g


def usp_set_wait_limit(ctx: Context, cycles: int):
    """Wait limit (SM cycles) of the homogeneous particle pass; 0 = default."""
    _check(lib().usp_set_wait_limit(ctx.h, int(cycles)), "usp_set_wait_limit")


def usp_wait_check(ctx: Context, cycles: int):
    """Enqueue a bounded wait on a barrier nothing completes (timeout check)."""
    _check(lib().usp_wait_check(ctx.h, int(cycles)), "usp_wait_check")


def usp_sync(ctx: Context):
    _check(lib().usp_sync(ctx.h), "usp_sync")


def usp_info(ctx: Context) -> dict:
    np_, st, b = C.c_int64(), C.c_int64(), C.c_int64()
    nc, pr, tl = C.c_int(), C.c_int(), C.c_int()
    _check(lib().usp_info(ctx.h, C.byref(np_), C.byref(nc), C.byref(pr), C.byref(st),
                          C.byref(tl), C.byref(b)), "usp_info")
    return dict(n_particles=np_.value, n_cells=nc.value, precision=pr.value, step=st.value,
                tile=tl.value, device_bytes=b.value)


def usp_tuning(ctx: Context):
    """(warp_tiles, blocks_per_sm) of the particle-pass variant in use and the
    autotuner's ms per launch [block-tiled 2, 3, 4, warp-tiled 2, 3, 4]."""
    wt = C.c_int()
    mb = C.c_int()
    ms = np.zeros(6)
    _check(lib().usp_tuning(ctx.h, C.byref(wt), C.byref(mb), _p(ms, C.c_double)), "usp_tuning")
    return (wt.value, mb.value), ms


def usp_set_variant(ctx: Context, warp_tiles: int, blocks_per_sm: int):
    """Force the particle-pass variant of a homogeneous context."""
    _check(lib().usp_set_variant(ctx.h, int(warp_tiles), int(blocks_per_sm)), "usp_set_variant")


def usp_launch_count(ctx: Context) -> int:
    return lib().usp_launch_count(ctx.h)


def usp_profile_enable(ctx: Context, on: bool = True):
    _check(lib().usp_profile_enable(ctx.h, 1 if on else 0), "usp_profile_enable")


def usp_profile_read(ctx: Context):
    """(ms[2], launches[2]) accumulated per kernel kind: 0 collide, 1 finalize."""
    ms = np.zeros(2)
    n = np.zeros(2, dtype=np.int64)
    _check(lib().usp_profile_read(ctx.h, _p(ms, C.c_double), _p(n, C.c_int64)), "usp_profile_read")
    return ms, n


def usp_moments_noalloc(species: dict, n_cells: int, d_offsets: int, d_cx: int, d_cy: int,
                        d_cz: int, d_erot: int, d_lev: int, d_out: int, stream: int = 0):
    """Per-cell moments of a device-resident state, without any device
    allocation (for callers whose memory is owned by their own pool).  All
    pointers are device addresses (ints); returns without waiting."""
    sp = make_species(species)
    rc = lib().usp_moments_noalloc(C.byref(sp), n_cells, *[C.c_void_p(x) for x in
                                   (d_offsets, d_cx, d_cy, d_cz, d_erot, d_lev, d_out)],
                                   C.c_void_p(stream or None))
    _check(rc, "usp_moments_noalloc")


def usp_destroy(ctx: Context):
    ctx.destroy()


def torch_allocator():
    """Allocator callbacks routing the library's device memory through
    PyTorch's caching allocator on the current device and stream."""
    import torch
    dev = torch.cuda.current_device()

    @ALLOC_FN
    def _alloc(nbytes, user):
        return torch.cuda.caching_allocator_alloc(int(nbytes), dev)

    @FREE_FN
    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    return _alloc, _free, None
