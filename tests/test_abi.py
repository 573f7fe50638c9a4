"""C-ABI library checks that need no GPU: it builds for sm_103a, loads, exports
every function declared in include/usp.h, and rejects invalid arguments on the
host before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2508_05642_gb300 import inputs as I
from paper_2508_05642_gb300 import usp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(usp_\w+)\s*\(", txt, flags=re.M):
                names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ["usp_init_homogeneous", "usp_step", "usp_moments", "usp_status", "usp_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    L = usp.lib()
    for name in _declared_functions():
        assert hasattr(L, name), name
    assert set(_declared_functions()) <= set(usp.EXPORTED) | {"usp_strerror"}


def test_strerror_and_tau_c_on_host():
    assert usp.usp_strerror(usp.USP_EINVAL) == "invalid argument"
    sp = I.n2_vhs_relaxation_species()
    # same closed form as the paper's Eq. tau_c; cfg-1 state
    assert usp.usp_tau_c(sp, 1e23, 1e4) == pytest.approx(1.1171e-8, rel=1e-4)


def test_invalid_arguments_rejected_before_device_work():
    sp = I.n2_vhs_relaxation_species()
    z = np.zeros(4)
    lev = np.zeros(4, dtype=np.int32)
    cases = [
        dict(offsets=[1, 4], ndens=[1e23], dt=[1e-9]),      # offsets[0] != 0
        dict(offsets=[0, 4, 2], ndens=[1e23] * 2, dt=[1e-9] * 2),  # decreasing
        dict(offsets=[0, 4], ndens=[0.0], dt=[1e-9]),       # density
        dict(offsets=[0, 4], ndens=[1e23], dt=[-1.0]),      # time step
    ]
    for c in cases:
        with pytest.raises(usp.USPError) as ei:
            usp.usp_init_homogeneous(sp, c["offsets"], c["ndens"], c["dt"], z, z, z, z, lev)
        assert ei.value.code == usp.USP_EINVAL
    with pytest.raises(usp.USPError) as ei:
        usp.usp_init_homogeneous(sp, [0, 4], [1e23], [1e-9], z, z, z, z, lev, precision=7)
    assert ei.value.code == usp.USP_EINVAL
    bad = dict(sp, m=0.0)
    with pytest.raises(usp.USPError):
        usp.usp_init_homogeneous(bad, [0, 4], [1e23], [1e-9], z, z, z, z, lev)


@pytest.mark.parametrize("levels,r2,r3,r", [(0, 0.0, 0.0, 0.1), (2, 0.3, 0.0, 0.0),
                                            (3, 0.3, 0.2, 0.1524), (3, 0.24, 0.155, 0.1524)])
def test_plane_leaves_on_the_host_match_the_oracle(levels, r2, r3, r):
    """The library's refined-grid layout (host code, no GPU) is the oracle's:
    same cells, levels and coordinates, in the same order; a grid whose
    neighbouring levels differ by two is rejected by both."""
    from oracle import oracle as O
    d = dict(nx=64, ny=48, x0=-0.4, x1=0.4, y0=0.0, y1=0.6, cyl_xc=0.0, cyl_yc=0.0, cyl_r=r,
             amr_levels=levels, amr_r2=r2, amr_r3=r3)
    lv, ii, jj = usp.usp_plane_leaves(dict(d, T_wall=500.0, n_inf=1e21, T_inf=200.0, U_inf=0.0,
                                           bc=(0, 0, 1, 0), inflow=(1, 0, 0, 1), F_num=1.0,
                                           depth=1.0, reconstruct=1), arrays=True)
    olv, oii, ojj = O.plane_leaves(O.plane(**d))
    for a, b in zip((lv, ii, jj), (olv, oii, ojj)):
        np.testing.assert_array_equal(a, b)
    bad = dict(d, amr_levels=3, amr_r2=0.2, amr_r3=0.2)
    assert O.plane_nleaf(O.plane(**bad)) == -1
    with pytest.raises(usp.USPError):
        usp.usp_plane_leaves(dict(bad, T_wall=500.0, n_inf=1e21, T_inf=200.0, U_inf=0.0,
                                  bc=(0, 0, 1, 0), inflow=(1, 0, 0, 1), F_num=1.0, depth=1.0,
                                  reconstruct=1))


class _CountingAllocator:
    """Allocator callbacks that hand out distinct fake addresses (never
    dereferenced: the library fails before any device work) and return NULL
    at the ``fail_at``-th request; they count what is outstanding."""

    def __init__(self, fail_at):
        self.fail_at = fail_at
        self.calls = 0
        self.live = set()

        @usp.ALLOC_FN
        def _alloc(nbytes, user):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = 0x7f0000000000 + 0x100000 * self.calls
            self.live.add(p)
            return p

        @usp.FREE_FN
        def _free(ptr, user):
            self.live.discard(ptr)

        self.fns = (_alloc, _free, None)


@pytest.mark.parametrize("precision", [usp.USP_FP32, usp.USP_FP64])
def test_failing_allocator_returns_enomem_and_frees_everything(precision):
    """A caller allocator that fails at any one request: context creation
    returns USP_ENOMEM before any CUDA call, having released through the free
    callback everything it had taken."""
    w = I.batched_instances(seed=2, n_inst=3, nmin=20, nmax=50, steps=1)
    dt = np.full(w.n_cells, 1e-9)
    p = w.particles
    probe = _CountingAllocator(fail_at=1)
    with pytest.raises(usp.USPError) as e:
        usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz, p.erot,
                                 p.lev, precision=precision, allocator=probe.fns)
    assert e.value.code == usp.USP_ENOMEM and not probe.live
    n_alloc = 0
    k = 1
    while True:
        a = _CountingAllocator(fail_at=k)
        try:
            usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz,
                                     p.erot, p.lev, precision=precision, allocator=a.fns)
        except usp.USPError as err:
            if err.code != usp.USP_ENOMEM:
                raise
            assert not a.live, (k, len(a.live))
            n_alloc = max(n_alloc, a.calls)
            k += 1
            if k > n_alloc:
                break
            continue
        raise AssertionError("context created on fake device memory")
    assert n_alloc >= 10


@pytest.mark.skipif(usp.lib().usp_select_device(0) == 0, reason="a GPU is present")
def test_allocator_memory_released_when_the_device_is_missing():
    """Every allocation succeeds, the first CUDA call fails (no device): the
    context is not created (USP_ECUDA) and nothing is left allocated."""
    w = I.batched_instances(seed=2, n_inst=3, nmin=20, nmax=50, steps=1)
    dt = np.full(w.n_cells, 1e-9)
    p = w.particles
    a = _CountingAllocator(fail_at=-1)
    with pytest.raises(usp.USPError) as e:
        usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz, p.erot,
                                 p.lev, precision=usp.USP_FP32, allocator=a.fns)
    assert e.value.code in (usp.USP_ECUDA, usp.USP_EINVAL)
    assert a.calls >= 10 and not a.live
