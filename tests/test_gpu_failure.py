"""Failure paths on the GPU, made without faulting or hanging it.

A wait that runs out: usp_wait_check makes the library's bounded wait run
on a barrier that nothing completes; the block must record
USP_F_WAIT_TIMEOUT and return, usp_status reports USP_EDEVICE on the host, and
the context stays usable.  The particle pass itself, given a one-cycle wait
limit, must return whatever its waits do.

A failing allocator: context creation with a caller allocator that returns
NULL at one request gives USP_ENOMEM and releases everything it had taken
through the free callback (real device memory here, from PyTorch's caching
allocator)."""
import numpy as np
import pytest

from paper_2508_05642_gb300 import inputs as I
from paper_2508_05642_gb300 import usp

pytestmark = pytest.mark.gpu


def _homog_ctx(precision=usp.USP_FP32, seed=4, n_inst=64):
    w = I.batched_instances(seed=seed, n_inst=n_inst, nmin=2000, nmax=20000, steps=5)
    dt = np.array([0.5 * usp.usp_tau_c(w.species, w.ndens[i], w.T_nominal[i, 0])
                   for i in range(w.n_cells)])
    p = w.particles
    return usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz, p.erot,
                                    p.lev, precision=precision, seed=w.seed, use_graph=False)


@pytest.mark.parametrize("kind", ["homogeneous", "channel"])
def test_wait_timeout_is_reported_and_the_context_stays_usable(kind):
    """usp_wait_check runs the library's bounded wait on a barrier that
    nothing completes, with a limit of 1e5 SM cycles: the block gives up,
    records USP_F_WAIT_TIMEOUT and returns; the host sees USP_EDEVICE; after a
    reset the context steps on, bit for bit as a twin that never waited."""
    if kind == "homogeneous":
        make = lambda: _homog_ctx(seed=8, n_inst=16)  # noqa: E731
    else:
        w = I.channel_poiseuille(ny=16, ppc=100, steps=0)
        dt = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.n, w.channel["T_wall"])
        p = w.particles
        make = lambda: usp.usp_init_channel(w.species, w.channel, dt, w.y, p.cx, p.cy, p.cz,  # noqa: E731
                                            p.erot, p.lev, precision=usp.USP_FP32, seed=3)
    ctx, twin = make(), make()
    usp.usp_step(ctx, 2)
    usp.usp_step(twin, 2)
    usp.usp_wait_check(ctx, 100000)
    flags, _ = usp.usp_status(ctx)
    assert flags & usp.F_WAIT_TIMEOUT
    assert usp.lib().usp_status(ctx.h, None, None, 1) == usp.USP_EDEVICE
    assert usp.lib().usp_status(ctx.h, None, None, 0) == usp.USP_OK
    usp.usp_step(ctx, 3)
    usp.usp_step(twin, 3)
    flags, _ = usp.usp_status(ctx)
    assert flags & usp.ERROR_FLAGS == 0
    get = usp.usp_get_particles if kind == "homogeneous" else usp.usp_channel_get_particles
    for x, y in zip(get(ctx), get(twin)):
        assert np.array_equal(x, y)
    ctx.destroy()
    twin.destroy()
    with pytest.raises(usp.USPError):
        c = make()
        try:
            usp.usp_wait_check(c, 0)
        finally:
            c.destroy()


def test_particle_pass_with_a_short_wait_limit_returns():
    """A wait limit of one cycle on the particle pass: whether or not a wait
    runs out (the hardware try-wait itself suspends for a while), the pass
    returns, a timeout is reported as USP_EDEVICE, and the device serves a
    new context cleanly afterwards."""
    for wt in (0, 1):
        ctx = _homog_ctx()
        usp.usp_set_variant(ctx, wt, 3)
        usp.usp_set_wait_limit(ctx, 1)
        usp.usp_step(ctx, 1)
        flags, _ = usp.usp_status(ctx)
        rc = usp.lib().usp_status(ctx.h, None, None, 1)
        assert rc == (usp.USP_EDEVICE if flags & usp.ERROR_FLAGS else usp.USP_OK)
        ctx.destroy()
    ok = _homog_ctx(seed=5)
    usp.usp_step(ok, 2)
    flags, _ = usp.usp_status(ok)
    assert flags & usp.ERROR_FLAGS == 0
    ok.destroy()


def test_default_wait_limit_restored():
    ctx = _homog_ctx(seed=6, n_inst=16)
    usp.usp_set_wait_limit(ctx, 1)
    usp.usp_set_wait_limit(ctx, 0)
    usp.usp_step(ctx, 2)
    flags, _ = usp.usp_status(ctx)
    assert flags & usp.F_WAIT_TIMEOUT == 0
    with pytest.raises(usp.USPError):
        usp.usp_set_wait_limit(ctx, -1)
    ctx.destroy()


class _TorchAllocator:
    """Caller allocator on PyTorch's caching allocator that returns NULL at
    the fail_at-th request and tracks what is outstanding."""

    def __init__(self, fail_at):
        import torch
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = set()
        dev = torch.cuda.current_device()

        @usp.ALLOC_FN
        def _alloc(nbytes, user):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev)
            self.live.add(p)
            return p

        @usp.FREE_FN
        def _free(ptr, user):
            self.live.discard(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        self.fns = (_alloc, _free, None)


def _count_requests(make):
    a = _TorchAllocator(fail_at=-1)
    ctx = make(a.fns)
    n = a.calls
    ctx.destroy()
    assert not a.live
    return n


@pytest.mark.parametrize("kind", ["homogeneous", "channel"])
def test_allocation_failure_at_every_request(kind):
    if kind == "homogeneous":
        w = I.batched_instances(seed=7, n_inst=8, nmin=200, nmax=2000, steps=1)
        dt = np.array([0.5 * usp.usp_tau_c(w.species, w.ndens[i], w.T_nominal[i, 0])
                       for i in range(w.n_cells)])
        p = w.particles

        def make(fns):
            return usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz,
                                            p.erot, p.lev, precision=usp.USP_FP32,
                                            allocator=fns)
    else:
        w = I.channel_poiseuille(ny=8, ppc=50, steps=0)
        dt = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.n, w.channel["T_wall"])
        p = w.particles

        def make(fns):
            return usp.usp_init_channel(w.species, w.channel, dt, w.y, p.cx, p.cy, p.cz, p.erot,
                                        p.lev, precision=usp.USP_FP64, allocator=fns)
    n = _count_requests(make)
    assert n >= 5
    for k in range(1, n + 1):
        a = _TorchAllocator(fail_at=k)
        with pytest.raises(usp.USPError) as e:
            make(a.fns)
        assert e.value.code == usp.USP_ENOMEM, k
        assert not a.live, (k, len(a.live))
