"""GPU parity of the spatial (1D channel) USP-FPM step against the FP64 oracle:
ballistic move with diffuse walls and body force, stable cell sort,
reconstruction (Sec. 3.B), per-particle collision and conservation, and the
time-average sums."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I
from paper_2508_05642_gb300 import usp

pytestmark = pytest.mark.gpu


def _pair(w, steps, precision, sample_last=0, use_graph=True):
    sp = O.species(**w.species)
    ch = O.channel(**w.channel)
    p = w.particles
    y = w.y
    form = 1 if precision == usp.USP_FP32 else 0
    if form == 1:
        p = p.astype_f32_exact()
        y = y.astype(np.float32).astype(np.float64)
    dto = w.dt_over_tau_c * O.tau_c(sp, w.n, w.channel["T_wall"])
    dtg = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.n, w.channel["T_wall"])
    st = O.ChannelState.from_arrays(y, p.cx, p.cy, p.cz, p.erot, p.lev)
    ctx = usp.usp_init_channel(w.species, w.channel, dtg, y, p.cx, p.cy, p.cz, p.erot, p.lev,
                               precision=precision, seed=w.seed, use_graph=use_graph)
    acc = np.zeros(ch.ny * O.NACC + 2)
    if steps - sample_last > 0:
        O.channel_step(sp, form, w.seed, 0, steps - sample_last, ch, dto, st)
        usp.usp_step(ctx, steps - sample_last)
    if sample_last:
        O.channel_step(sp, form, w.seed, steps - sample_last, sample_last, ch, dto, st, acc)
        usp.usp_channel_sample(ctx, True)
        usp.usp_step(ctx, sample_last)
    g = usp.usp_channel_get_particles(ctx)
    gacc = usp.usp_channel_read(ctx)
    gfl, gcnt = usp.usp_status(ctx)
    return dict(sp=sp, ch=ch, st=st, g=g, acc=acc, gacc=gacc, gfl=gfl, gcnt=gcnt, ctx=ctx)


def test_fp64_channel_full_size_100_steps_matches_oracle():
    """The Poiseuille workload at its full size (64 cells x 200 particles)
    over its first 100 steps, the last 20 sampled: same particles in the same
    cell order, same levels, values within FP64 rounding, same time-average
    sums.  (The runs stay one realization for about 500 steps: their velocity
    difference grows tenfold per 100 steps from rounding size.)"""
    w = I.channel_poiseuille(ny=64, ppc=200, steps=0)
    r = _pair(w, 100, usp.USP_FP64, sample_last=20)
    st, (gy, gx, gyv, gz, ge, gl, gp) = r["st"], r["g"]
    R = O.R(r["sp"])
    vth = math.sqrt(R * 300.0)
    assert np.array_equal(gp, st.pid) and np.array_equal(gl, st.lev)
    assert np.max(np.abs(gy - st.y)) < 1e-9 * r["ch"].L
    for a, b in ((gx, st.cx), (gyv, st.cy), (gz, st.cz)):
        assert np.max(np.abs(a - b)) < 1e-8 * vth
    assert np.max(np.abs(ge - st.erot)) < 1e-8 * R * 300.0
    np.testing.assert_allclose(r["gacc"], r["acc"], rtol=1e-9, atol=1e-6)
    assert r["gcnt"][usp.C_WALL_HITS] > 0 and r["gfl"] & usp.ERROR_FLAGS == 0


def test_fp64_channel_matches_oracle_step_by_step():
    w = I.channel_poiseuille(ny=16, ppc=100, steps=0)
    r = _pair(w, 30, usp.USP_FP64, sample_last=10)
    st, (gy, gx, gyv, gz, ge, gl, gp) = r["st"], r["g"]
    R = O.R(r["sp"])
    vth = math.sqrt(R * 300.0)
    assert np.array_equal(gp, st.pid)          # same stable cell order
    assert np.array_equal(gl, st.lev)
    assert np.max(np.abs(gy - st.y)) < 1e-9 * r["ch"].L
    for a, b in ((gx, st.cx), (gyv, st.cy), (gz, st.cz)):
        assert np.max(np.abs(a - b)) < 1e-8 * vth
    assert np.max(np.abs(ge - st.erot)) < 1e-8 * R * 300.0
    np.testing.assert_allclose(r["gacc"], r["acc"], rtol=1e-9, atol=1e-6)
    assert r["gcnt"][usp.C_WALL_HITS] > 0


def test_fp32_channel_single_step_matches_oracle():
    """192,000 particles, one step from the identical FP32 state: per-particle
    values within FP32 rounding of the arithmetic, level mismatches < 1e-5."""
    w = I.channel_poiseuille(ny=64, ppc=3000, steps=0)
    r = _pair(w, 1, usp.USP_FP32)
    st, (gy, gx, gyv, gz, ge, gl, gp) = r["st"], r["g"]
    o = np.argsort(st.pid)
    gpo = np.argsort(gp)
    R = O.R(r["sp"])
    vth = math.sqrt(R * 300.0)
    assert np.mean(gl[gpo] != st.lev[o]) < 1e-5
    dv = np.abs(gx[gpo] - st.cx[o])
    assert np.quantile(dv, 0.999) < 2e-5 * vth and np.max(dv) < 1e-3 * vth
    # float positions: a few ulps of y ~ L (far below a cell width, L / 64)
    assert np.max(np.abs(gy[gpo] - st.y[o])) < 1e-5 * r["ch"].L
    de = np.abs(ge[gpo] - st.erot[o])
    assert np.quantile(de, 0.999) < 1e-4 * R * 300.0


def test_channel_graph_and_eager_agree():
    w = I.channel_poiseuille(ny=16, ppc=50, steps=0)
    outs = []
    for g in (True, False):
        ctx = usp.usp_init_channel(w.species, w.channel,
                                   0.2 * usp.usp_tau_c(w.species, w.n, 300.0), w.y,
                                   w.particles.cx, w.particles.cy, w.particles.cz,
                                   w.particles.erot, w.particles.lev, precision=usp.USP_FP32,
                                   seed=3, use_graph=g)
        usp.usp_step(ctx, 40)
        outs.append(usp.usp_channel_get_particles(ctx))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_fp32_poiseuille_matches_oracle_profile():
    """Developed force-driven Poiseuille flow: the FP32 GPU runs' time-averaged
    velocity profile agrees with the FP64 oracle's within the statistical
    scatter, and both balance the body force with wall friction.  Different
    seeds are different realizations: the centreline velocity of one
    5,000-step average scatters by about 3.5 % between seeds, so the test
    compares means over six library seeds and three oracle seeds (standard
    error of the difference about 2.3 %) at 8 %."""
    w = I.channel_poiseuille(ny=32, ppc=100, steps=0)
    sp = O.species(**w.species)
    ch = O.channel(**w.channel)
    dto = w.dt_over_tau_c * O.tau_c(sp, w.n, 300.0)
    dtg = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.n, 300.0)
    p = w.particles
    n = len(w.y)
    force = n * ch.g * dto

    def profile(a):
        A = a[: ch.ny * O.NACC].reshape(ch.ny, O.NACC)
        return A[:, 1] / A[:, 0]

    uo = []
    for seed in (11, 21, 31):
        st = O.ChannelState.from_arrays(w.y, p.cx, p.cy, p.cz, p.erot, p.lev)
        O.channel_step(sp, 0, seed, 0, 2000, ch, dto, st)
        acc = np.zeros(ch.ny * O.NACC + 2)
        O.channel_step(sp, 0, seed, 2000, 5000, ch, dto, st, acc)
        assert acc[-1] / 5000 == pytest.approx(force, rel=0.03)
        uo.append(profile(acc))
    ug = []
    for seed in (12, 13, 14, 15, 16, 17):
        ctx = usp.usp_init_channel(w.species, w.channel, dtg, w.y, p.cx, p.cy, p.cz, p.erot,
                                   p.lev, precision=usp.USP_FP32, seed=seed)
        usp.usp_step(ctx, 2000)
        usp.usp_channel_sample(ctx, True)
        usp.usp_step(ctx, 5000)
        gacc = usp.usp_channel_read(ctx)
        flags, cnt = usp.usp_status(ctx)
        ctx.destroy()
        # clamps of relaxation temperatures occur where the sparse vibrational
        # excitation (mean level ~1e-5 at 300 K) makes the cell T_vib jump;
        # only error bits fail the run
        assert flags & usp.ERROR_FLAGS == 0
        assert gacc[-1] / 5000 == pytest.approx(force, rel=0.03)
        ug.append(profile(gacc))
    uo, ug = np.mean(uo, axis=0), np.mean(ug, axis=0)
    mid = slice(ch.ny // 2 - 4, ch.ny // 2 + 4)
    assert ug[mid].mean() == pytest.approx(uo[mid].mean(), rel=0.08)
    assert np.abs(ug - uo).max() < 0.15 * uo.max()
