"""GPU test of usp_moments_noalloc, the entry point for callers that may not
allocate device memory (for example a framework that owns all device memory
in its own pool, or a time loop that must not hit the implicit
synchronisation of cudaMalloc/cudaFree).  It must give the same per-cell
moments as usp_moments of a context holding the same particles, call after
call, while the only device memory it touches besides the caller's buffers is
its fixed in-library scratch array.

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test first; it also passes on its own in a fresh
process.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I
from paper_2508_05642_gb300 import usp

pytestmark = pytest.mark.gpu


def _close(a, ref, rel=1e-5):
    """Same bar as the moment parity tests: 1e-5 relative to each field's scale."""
    for f in range(ref.shape[0]):
        scale = max(np.abs(ref[f]).max(), 1e-300)
        assert np.all(np.abs(a[f] - ref[f]) <= rel * np.maximum(np.abs(ref[f]), scale)), f


def test_noalloc_moments_match_context_moments_twice():
    torch = pytest.importorskip("torch")
    w = I.batched_instances(seed=21, n_inst=300, nmin=100, nmax=20000, steps=0)
    p = w.particles
    dt = np.array([0.5 * usp.usp_tau_c(w.species, w.ndens[i], w.T_nominal[i, 0])
                   for i in range(w.n_cells)])
    ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz, p.erot,
                                   p.lev, precision=usp.USP_FP64, seed=3)
    usp.usp_step(ctx, 3)
    ref = usp.usp_moments(ctx)
    cx, cy, cz, er, lv = usp.usp_get_particles(ctx)
    ctx.destroy()

    dev = torch.device("cuda", torch.cuda.current_device())
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    dcx, dcy, dcz, der = d(cx), d(cy), d(cz), d(er)
    dlv = d(lv.astype(np.int32))
    doff = d(w.offsets.astype(np.int64))
    out = torch.empty((usp.USP_NMOM, w.n_cells), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    # the oracle's moments of the same particles, cell by cell
    orc = O.moments(O.species(**w.species), w.offsets, O.State.from_arrays(cx, cy, cz, er, lv))
    for k in range(2):
        out.fill_(np.nan)
        torch.cuda.synchronize()
        if k == 1:
            free0 = torch.cuda.mem_get_info()[0]
            alloc0 = torch.cuda.memory_allocated()
        usp.usp_moments_noalloc(w.species, w.n_cells, doff.data_ptr(), dcx.data_ptr(),
                                dcy.data_ptr(), dcz.data_ptr(), der.data_ptr(), dlv.data_ptr(),
                                out.data_ptr(), stream)
        torch.cuda.synchronize()
        if k == 1:
            # the second call took no device memory from the driver or torch
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
        got = out.cpu().numpy()
        _close(got, ref)
        # per cell, against the oracle (1e-5 relative to each cell's value,
        # with a floor of 1e-9 of the field's scale for values near zero)
        for f in range(orc.shape[0]):
            scale = max(np.abs(orc[f]).max(), 1e-300)
            assert np.all(np.abs(got[f] - orc[f]) <= 1e-5 * np.abs(orc[f]) + 1e-9 * scale), f


def test_noalloc_rejects_more_cells_than_its_scratch_holds():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", torch.cuda.current_device())
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    lv = torch.zeros(16, dtype=torch.int32, device=dev)
    off = torch.zeros(16, dtype=torch.int64, device=dev)
    with pytest.raises(usp.USPError) as ei:
        usp.usp_moments_noalloc(I.n2_vhs_relaxation_species(), usp.USP_NOALLOC_MAX_CELLS + 1,
                                off.data_ptr(), buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                buf.data_ptr(), lv.data_ptr(), buf.data_ptr(), 0)
    assert ei.value.code == usp.USP_EINVAL
