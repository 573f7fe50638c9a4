"""GPU parity of the plain FPM method (Sec. 2.B model, Sec. 2.C scheme:
Gorji's velocity integrator, the modified-Milstein rotational update,
Gillespie's direct method for the levels, the conservation scheme of
Sec. 4.C) against the oracle's FPM method on the same seeded inputs, with the
bars of the USP-FPM parity tests."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I
from paper_2508_05642_gb300 import usp
from test_gpu_homog import _check_moments, _gpu_dt, _oracle_dt

pytestmark = pytest.mark.gpu


def _ragged(seed, n_inst, nmin, nmax, steps, small=True):
    w = I.batched_instances(seed=seed, n_inst=n_inst, nmin=nmin, nmax=nmax, steps=steps)
    if not small:
        return w
    counts = np.diff(w.offsets)
    counts[:4] = [0, 1, 2, 3]
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    rng = np.random.default_rng(seed + 1)
    sp = w.species
    parts = [I.equilibrium_particles(rng, int(n), sp["m"], sp["theta_v"], T_tr=w.T_nominal[i, 0],
                                     T_rot=w.T_nominal[i, 1], T_vib=w.T_nominal[i, 2])
             for i, n in enumerate(counts)]
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])
    w.offsets = off
    w.particles = I.Particles(cat("cx"), cat("cy"), cat("cz"), cat("erot"), cat("lev"))
    return w


def _run(w, steps, precision, **kw):
    form = 1 if precision == usp.USP_FP32 else 0
    p = w.particles.astype_f32_exact() if form else w.particles
    st = O.State.from_arrays(p.cx, p.cy, p.cz, p.erot, p.lev)
    sp = O.species(**w.species)
    ofl, _ = O.homog_step_fpm(sp, form, w.seed, 0, steps, w.offsets, w.ndens, _oracle_dt(w), st)
    ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, _gpu_dt(w), p.cx, p.cy, p.cz,
                                   p.erot, p.lev, precision=precision, seed=w.seed,
                                   method=usp.USP_METHOD_FPM, **kw)
    return ctx, st, sp, ofl


def test_fpm_fp64_batched_ragged_matches_oracle():
    """FP64 form, ten steps, 40 cells of uneven size (0 to 3000 particles,
    several tiles with ragged tails); cells of fewer than two particles stay
    untouched."""
    w = _ragged(31, 40, 50, 3000, 10)
    ctx, st, sp, ofl = _run(w, 10, usp.USP_FP64, tile=256)
    usp.usp_step(ctx, 10)
    gm = usp.usp_moments(ctx)
    gs = usp.usp_get_particles(ctx)
    fl, _ = usp.usp_status(ctx)
    assert fl & usp.ERROR_FLAGS == 0 and ofl & O.F_SAMPLER_CAP == 0
    om = O.moments(sp, w.offsets, st)
    _check_moments(om, gm, sp)
    assert np.mean(gs[4] != st.lev) < 1e-5
    for i in range(2):
        b, e = w.offsets[i], w.offsets[i + 1]
        assert np.array_equal(gs[0][b:e], w.particles.cx[b:e])


def test_fpm_fp32_single_step_matches_oracle():
    """FP32 state, one step from the identical state; the Gillespie decisions
    are taken in float on both sides."""
    w = _ragged(33, 24, 500, 20000, 1, small=False)
    ctx, st, sp, _ = _run(w, 1, usp.USP_FP32, tile=1024)
    usp.usp_step(ctx, 1)
    gm = usp.usp_moments(ctx)
    gx, gy, gz, ge, gl = usp.usp_get_particles(ctx)
    om = O.moments(sp, w.offsets, st)
    _check_moments(om, gm, sp)
    assert np.mean(gl != st.lev) < 1e-4
    R = O.R(sp)
    for i in range(w.n_cells):
        b, e = w.offsets[i], w.offsets[i + 1]
        vth = math.sqrt(R * om[4, i])
        assert np.max(np.abs(gx[b:e] - st.cx[b:e])) < 2e-5 * vth
        assert np.max(np.abs(gz[b:e] - st.cz[b:e])) < 2e-5 * vth


@pytest.mark.parametrize("wt,mb", [(0, 2), (0, 3), (0, 4), (1, 2), (1, 3), (1, 4)])
def test_fpm_every_particle_pass_variant(wt, mb):
    """Both particle-pass designs at each register budget, FP64 form, four
    steps, against one oracle run."""
    w = _ragged(35, 30, 2, 6000, 4, small=False)
    ctx, st, sp, _ = _run(w, 4, usp.USP_FP64)
    usp.usp_set_variant(ctx, wt, mb)
    usp.usp_step(ctx, 4)
    gm = usp.usp_moments(ctx)
    gl = usp.usp_get_particles(ctx)[4]
    fl, _ = usp.usp_status(ctx)
    assert fl & usp.ERROR_FLAGS == 0
    _check_moments(O.moments(sp, w.offsets, st), gm, sp)
    assert np.mean(gl != st.lev) < 1e-5


def test_fpm_conservation_on_gpu_fp64():
    """Sec. 4.C with the FPM method on the GPU: per-cell momentum and total
    energy conserved to FP64 rounding over ten steps."""
    w = _ragged(37, 12, 200, 5000, 10, small=False)
    p = w.particles
    ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, _gpu_dt(w), p.cx, p.cy, p.cz,
                                   p.erot, p.lev, precision=usp.USP_FP64, seed=3,
                                   method=usp.USP_METHOD_FPM)
    sp = O.species(**w.species)
    Rth = O.R(sp) * sp.theta_v
    def totals(cx, cy, cz, er, lv):
        out = []
        for i in range(w.n_cells):
            b, e = w.offsets[i], w.offsets[i + 1]
            out.append((np.array([cx[b:e].sum(), cy[b:e].sum(), cz[b:e].sum()]),
                        (0.5 * (cx[b:e] ** 2 + cy[b:e] ** 2 + cz[b:e] ** 2) + er[b:e]
                         + Rth * lv[b:e]).sum(),
                        np.sqrt((cx[b:e] ** 2).sum())))
        return out
    t0 = totals(p.cx, p.cy, p.cz, p.erot, p.lev)
    usp.usp_step(ctx, 10)
    t1 = totals(*usp.usp_get_particles(ctx))
    for (m0, e0, v0), (m1, e1, _) in zip(t0, t1):
        assert np.max(np.abs(m1 - m0)) <= 1e-11 * v0
        assert e1 == pytest.approx(e0, rel=1e-12)


# ---- the plain FPM method on the plane path (cell values) -------------------
def _plane_pair(w, steps, precision, seed=3):
    from oracle import oracle as Oo
    sp = Oo.species(**w.species)
    dto = w.dt_over_tau_c * Oo.tau_c(sp, w.plane["n_inf"], w.plane["T_inf"])
    dtg = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.plane["n_inf"], w.plane["T_inf"])
    pl = Oo.plane(**dict(w.plane, method=1))
    p = w.particles
    form = 1 if precision == usp.USP_FP32 else 0
    st = Oo.PlaneState(w.x, w.y, p.cx, p.cy, p.cz, p.erot, p.lev, w.capacity)
    ctx = usp.usp_init_plane(w.species, w.plane, dtg, w.area_frac, w.x, w.y, p.cx, p.cy, p.cz,
                             p.erot, p.lev, w.capacity, precision=precision, seed=seed,
                             method=usp.USP_METHOD_FPM)
    _, fl, cnt = Oo.plane_step(sp, form, seed, 0, steps, pl, w.area_frac, dto, st)
    usp.usp_step(ctx, steps)
    g = usp.usp_plane_get_particles(ctx)
    gfl, gcnt = usp.usp_status(ctx)
    return sp, st, g, cnt, gfl, gcnt


@pytest.mark.parametrize("refined", [False, True])
def test_fp64_plane_fpm_matches_oracle(refined):
    """The cylinder with the plain FPM method (FP64 form), 16 steps on the
    uniform 48 x 32 grid and on a three-level grid: same particles in the same
    order, same levels (Gillespie), values within FP64 rounding of the
    arithmetic, same inflow / outflow / wall-event counts."""
    from oracle import oracle as Oo
    kw = dict(amr_levels=3, amr_r2=0.22, amr_r3=0.14) if refined else {}
    w = I.cylinder_flow(nx=48 if not refined else 32, ny=32 if not refined else 24, ppc=12, **kw)
    sp, st, g, cnt, gfl, gcnt = _plane_pair(w, 16, usp.USP_FP64)
    gx, gy, gvx, gvy, gvz, ge, gl, gp = g
    assert len(gp) == st.n and np.array_equal(gp, st.pid[:st.n])
    assert np.array_equal(gl, st.lev[:st.n])
    R = Oo.R(sp)
    vth = math.sqrt(R * 200.0)
    assert np.max(np.abs(gx - st.x[:st.n])) < 1e-9
    for a, b in ((gvx, st.cx), (gvy, st.cy), (gvz, st.cz)):
        assert np.max(np.abs(a - b[:st.n])) < 1e-7 * vth
    assert np.max(np.abs(ge - st.erot[:st.n])) < 1e-7 * R * 200.0
    for k in (usp.C_INFLOW, usp.C_OUTFLOW, usp.C_WALL_HITS):
        assert gcnt[k] == cnt[k], k
    assert gfl & usp.ERROR_FLAGS == 0


def test_fp32_plane_fpm_levels_and_fields_track_the_oracle():
    """FP32 FPM plane against the FP32-form oracle over 12 steps of the small
    cylinder: bookkeeping identical, levels equal for all but a few particles
    (Gillespie decisions in float), velocities within FP32 arithmetic."""
    from oracle import oracle as Oo
    w = I.cylinder_flow(nx=48, ny=32, ppc=12)
    p = w.particles
    rnd = lambda a: a.astype(np.float32).astype(np.float64)
    w.particles = type(p)(cx=rnd(p.cx), cy=rnd(p.cy), cz=rnd(p.cz), erot=rnd(p.erot), lev=p.lev)
    w.x = np.clip(rnd(w.x), np.nextafter(np.float32(w.plane["x0"]), np.float32(1)),
                  np.nextafter(np.float32(w.plane["x1"]), np.float32(-1)))
    w.y = np.clip(rnd(w.y), w.plane["y0"], w.plane["y1"])
    sp, st, g, cnt, gfl, gcnt = _plane_pair(w, 12, usp.USP_FP32)
    gx, gy, gvx, gvy, gvz, ge, gl, gp = g
    assert gfl & usp.ERROR_FLAGS == 0
    assert len(gp) == st.n
    go, oo = np.argsort(gp), np.argsort(st.pid[:st.n])
    assert np.array_equal(gp[go], st.pid[:st.n][oo])
    assert np.mean(gl[go] != st.lev[:st.n][oo]) < 2e-3
    vth = math.sqrt(Oo.R(sp) * 200.0)
    dv = np.abs(gvx[go] - st.cx[:st.n][oo])
    assert np.quantile(dv, 0.99) < 1e-3 * vth


@pytest.mark.parametrize("precision", [usp.USP_FP64, usp.USP_FP32])
def test_channel_fpm_matches_oracle(precision):
    """The Poiseuille channel (16 cells x 100 particles) with the plain FPM
    method, 30 steps: FP64 form particle for particle (ids, order, levels,
    values within FP64 rounding of the arithmetic); FP32 form against the
    FP32-form oracle (levels equal for all but a few, velocities within FP32
    arithmetic at the 99th percentile); same wall-event counts in FP64."""
    from oracle import oracle as Oo
    w = I.channel_poiseuille(ny=16, ppc=100, steps=0)
    sp = Oo.species(**w.species)
    ch = Oo.channel(**dict(w.channel, method=1))
    p = w.particles
    y = w.y
    form = 1 if precision == usp.USP_FP32 else 0
    if form == 1:
        p = p.astype_f32_exact()
        y = y.astype(np.float32).astype(np.float64)
    dto = w.dt_over_tau_c * Oo.tau_c(sp, w.n, w.channel["T_wall"])
    dtg = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.n, w.channel["T_wall"])
    st = Oo.ChannelState.from_arrays(y, p.cx, p.cy, p.cz, p.erot, p.lev)
    ctx = usp.usp_init_channel(w.species, w.channel, dtg, y, p.cx, p.cy, p.cz, p.erot, p.lev,
                               precision=precision, seed=w.seed, method=usp.USP_METHOD_FPM)
    _, fl, cnt = Oo.channel_step(sp, form, w.seed, 0, 30, ch, dto, st)
    usp.usp_step(ctx, 30)
    gy, gvx, gvy, gvz, ge, gl, gp = usp.usp_channel_get_particles(ctx)
    gfl, gcnt = usp.usp_status(ctx)
    assert gfl & usp.ERROR_FLAGS == 0
    vth = math.sqrt(Oo.R(sp) * 300.0)
    if form == 0:
        assert np.array_equal(gp, st.pid) and np.array_equal(gl, st.lev)
        assert np.max(np.abs(gy - st.y)) < 1e-12
        for a, b in ((gvx, st.cx), (gvy, st.cy), (gvz, st.cz)):
            assert np.max(np.abs(a - b)) < 1e-7 * vth
        assert gcnt[usp.C_WALL_HITS] == cnt[Oo.C_WALL_HITS]
    else:
        go, oo = np.argsort(gp), np.argsort(st.pid)
        assert np.array_equal(gp[go], st.pid[oo])
        assert np.mean(gl[go] != st.lev[oo]) < 2e-3
        assert np.quantile(np.abs(gvx[go] - st.cx[oo]), 0.99) < 1e-3 * vth
    with pytest.raises(usp.USPError):
        usp.usp_init_channel(w.species, w.channel, dtg, y, p.cx, p.cy, p.cz, p.erot, p.lev,
                             precision=usp.USP_FP64_TANGENT, method=usp.USP_METHOD_FPM)
