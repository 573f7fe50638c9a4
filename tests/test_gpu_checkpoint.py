"""Checkpoint / resume through the C ABI (usp_checkpoint_bytes, usp_save,
usp_load): a context restored from a checkpoint continues as the one that
saved it, with host and with device buffers; a checkpoint of another kind of
context is refused and leaves the context unchanged.

Bit for bit where the step is: the FP32 form's FP64 cell sums add FP32
values, exactly, in any order, and the channel reduces each cell in one warp.
The FP64 homogeneous form adds FP64 values from several warps per cell with
FP64 atomics, whose order varies between launches, so there the resumed run
agrees to rounding (1e-12 relative) with the same levels."""
import numpy as np
import pytest

from paper_2508_05642_gb300 import inputs as I
from paper_2508_05642_gb300 import usp

pytestmark = pytest.mark.gpu


def _homog(precision):
    w = I.batched_instances(seed=3, n_inst=12, nmin=300, nmax=3000, steps=20)
    dt = np.array([0.5 * usp.usp_tau_c(w.species, w.ndens[i], w.T_nominal[i, 0])
                   for i in range(w.n_cells)])
    p = w.particles
    return lambda: usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz,
                                            p.erot, p.lev, precision=precision, seed=w.seed)


@pytest.mark.parametrize("precision", [usp.USP_FP32, usp.USP_FP64])
@pytest.mark.parametrize("on_device", [False, True])
def test_homogeneous_resume_is_bitwise(precision, on_device):
    make = _homog(precision)
    a = make()
    usp.usp_step(a, 7)
    if on_device:
        import torch
        buf = torch.zeros(usp.usp_checkpoint_bytes(a), dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        usp.usp_save(a, buf.data_ptr(), buf_is_device=True)
        usp.usp_sync(a)
    else:
        buf = usp.usp_save(a)
    usp.usp_step(a, 9)
    ref = usp.usp_get_particles(a)
    ref_m = usp.usp_moments(a)
    b = make()
    usp.usp_step(b, 3)   # a different state, overwritten by the load
    if on_device:
        usp.usp_load(b, buf.data_ptr(), buf_is_device=True)
    else:
        usp.usp_load(b, buf)
    assert usp.usp_info(b)["step"] == 7
    usp.usp_step(b, 9)
    got = usp.usp_get_particles(b)
    if precision == usp.USP_FP32:
        for x, y in zip(ref, got):
            assert np.array_equal(x, y)
        assert np.array_equal(ref_m, usp.usp_moments(b))
    else:
        for x, y in zip(ref[:4], got[:4]):
            np.testing.assert_allclose(y, x, rtol=1e-12, atol=1e-12 * np.abs(x).max())
        assert np.array_equal(ref[4], got[4])
        got_m = usp.usp_moments(b)
        for f in range(ref_m.shape[0]):
            np.testing.assert_allclose(got_m[f], ref_m[f], rtol=1e-11,
                                       atol=1e-11 * np.abs(ref_m[f]).max())
    a.destroy()
    b.destroy()


def test_channel_resume_is_bitwise_with_sampling():
    w = I.channel_poiseuille(ny=16, ppc=100, steps=0)
    dt = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.n, w.channel["T_wall"])
    p = w.particles

    def make():
        return usp.usp_init_channel(w.species, w.channel, dt, w.y, p.cx, p.cy, p.cz, p.erot,
                                    p.lev, precision=usp.USP_FP32, seed=5)
    a = make()
    usp.usp_step(a, 5)
    usp.usp_channel_sample(a, True)
    usp.usp_step(a, 6)
    buf = usp.usp_save(a)
    usp.usp_step(a, 11)
    ref_acc = usp.usp_channel_read(a)
    ref_p = usp.usp_channel_get_particles(a)
    b = make()
    usp.usp_load(b, buf)
    usp.usp_step(b, 11)
    assert np.array_equal(ref_acc, usp.usp_channel_read(b))
    for x, y in zip(ref_p, usp.usp_channel_get_particles(b)):
        assert np.array_equal(x, y)
    a.destroy()
    b.destroy()


def test_foreign_checkpoint_is_refused():
    a = _homog(usp.USP_FP32)()
    b = _homog(usp.USP_FP64)()
    buf = usp.usp_save(b)
    before = usp.usp_get_particles(a)
    with pytest.raises(usp.USPError) as e:
        usp.usp_load(a, buf)
    assert e.value.code == usp.USP_EINVAL
    bad = usp.usp_save(a)
    bad[:4] = 0   # not a checkpoint header
    with pytest.raises(usp.USPError):
        usp.usp_load(a, bad)
    for x, y in zip(before, usp.usp_get_particles(a)):
        assert np.array_equal(x, y)
    a.destroy()
    b.destroy()
