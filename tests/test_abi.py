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
