"""GPU parity of the plane step on the refined grid (the three-level mesh of
Sec. 5.C, reconstruction over finer and coarser neighbours of Sec. 3.B)
against the FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I
from paper_2508_05642_gb300 import usp

pytestmark = pytest.mark.gpu


def _small(ppc=32, seed=1):
    # 32 x 24 level-1 cells, level 2 within 0.22 m, level 3 within 0.14 m of a
    # 0.1 m cylinder
    return I.cylinder_flow(nx=32, ny=24, ppc=ppc, amr_levels=3, amr_r2=0.22, amr_r3=0.14,
                           seed=seed)


def _dts(w):
    sp = O.species(**w.species)
    dto = w.dt_over_tau_c * O.tau_c(sp, w.plane["n_inf"], w.plane["T_inf"])
    dtg = w.dt_over_tau_c * usp.usp_tau_c(w.species, w.plane["n_inf"], w.plane["T_inf"])
    return sp, dto, dtg


def _inside32(a, lo, hi):
    """a rounded to float, kept within [lo, hi] (a bound itself may round
    outward)."""
    f = a.astype(np.float32)
    l32, h32 = np.float32(lo), np.float32(hi)
    if float(l32) < lo:
        l32 = np.nextafter(l32, np.float32(np.inf))
    if float(h32) > hi:
        h32 = np.nextafter(h32, np.float32(-np.inf))
    return np.clip(f, l32, h32).astype(np.float64)


def _state(w, f32=False):
    p = w.particles
    arr = [w.x, w.y, p.cx, p.cy, p.cz, p.erot]
    if f32:
        pl = w.plane
        arr = [_inside32(w.x, pl["x0"], pl["x1"]), _inside32(w.y, pl["y0"], pl["y1"])] + \
            [a.astype(np.float32).astype(np.float64) for a in arr[2:]]
    return arr + [p.lev]


def _leaf_of32(plane, x, y):
    """The FP32 state's point location, emulated in float arithmetic: the
    level-1 cell from (x - x0) / dx, then the half and the quarter of it from
    the offset in units of half a cell, as the library computes them; the
    cell index from the library's cell list (level, ii, jj)."""
    lv, ii, jj = usp.usp_plane_leaves(plane, arrays=True)
    key = (lv.astype(np.int64) << 44) | (jj.astype(np.int64) << 22) | ii.astype(np.int64)
    order = np.argsort(key)
    skey = key[order]

    def find(L, i, j):
        k = (np.int64(L) << 44) | (j.astype(np.int64) << 22) | i.astype(np.int64)
        pos = np.clip(np.searchsorted(skey, k), 0, len(skey) - 1)
        return np.where(skey[pos] == k, order[pos], -1)

    f = np.float32
    nx, ny = plane["nx"], plane["ny"]
    x, y = x.astype(f), y.astype(f)
    x0, y0 = f(plane["x0"]), f(plane["y0"])
    dx, dy = f((plane["x1"] - plane["x0"]) / nx), f((plane["y1"] - plane["y0"]) / ny)
    i = np.clip(np.floor((x - x0) / dx), 0, nx - 1).astype(np.int64)
    j = np.clip(np.floor((y - y0) / dy), 0, ny - 1).astype(np.int64)
    out = find(1, i, j)
    m = out < 0                                  # split level-1 cells
    ux = (x[m] - (x0 + i[m].astype(f) * dx)) / (f(0.5) * dx)
    uy = (y[m] - (y0 + j[m].astype(f) * dy)) / (f(0.5) * dy)
    ci, cj = (ux >= f(1)).astype(np.int64), (uy >= f(1)).astype(np.int64)
    i2, j2 = 2 * i[m] + ci, 2 * j[m] + cj
    l2 = find(2, i2, j2)
    vx, vy = (ux - ci.astype(f)) * f(2), (uy - cj.astype(f)) * f(2)
    l3 = find(3, 2 * i2 + (vx >= f(1)), 2 * j2 + (vy >= f(1)))
    out[m] = np.where(l2 >= 0, l2, l3)
    assert np.all(out >= 0)
    return out


def _pair(w, steps, precision, sample_last=0, seed=None):
    seed = w.seed if seed is None else seed
    sp, dto, dtg = _dts(w)
    pl = O.plane(**w.plane)
    form = 1 if precision == usp.USP_FP32 else 0
    x, y, cx, cy, cz, er, lev = _state(w, form == 1)
    st = O.PlaneState(x, y, cx, cy, cz, er, lev, w.capacity)
    ctx = usp.usp_init_plane(w.species, w.plane, dtg, w.area_frac, x, y, cx, cy, cz, er, lev,
                             w.capacity, precision=precision, seed=seed)
    acc = O.plane_acc(pl)
    cnt = np.zeros(O.NCOUNTERS, dtype=np.int64)
    if steps - sample_last > 0:
        _, f1, c1 = O.plane_step(sp, form, seed, 0, steps - sample_last, pl, w.area_frac, dto, st)
        cnt += c1
        usp.usp_step(ctx, steps - sample_last)
    off = None
    if sample_last:
        off, f2, c2 = O.plane_step(sp, form, seed, steps - sample_last, sample_last, pl,
                                   w.area_frac, dto, st, acc)
        cnt += c2
        usp.usp_sample(ctx, True)
        usp.usp_step(ctx, sample_last)
    g = usp.usp_plane_get_particles(ctx)
    gacc = usp.usp_sample_read(ctx)
    gfl, gcnt = usp.usp_status(ctx)
    return dict(sp=sp, pl=pl, st=st, g=g, acc=acc, gacc=gacc, gfl=gfl, gcnt=gcnt, cnt=cnt,
                ctx=ctx, off=off)


def test_fp64_refined_plane_matches_oracle_step_by_step():
    """32 x 24 level-1 cells on three levels (1,600-odd cells), ~24k particles,
    24 steps while the bow shock forms: same particles in the same order (so
    the same cell of every particle), same levels, values within FP64 rounding
    of the arithmetic, same per-cell time averages and surface tallies, same
    inflow / outflow / wall-event counts."""
    w = _small()
    lv = usp.usp_plane_leaves(w.plane, arrays=True)[0]
    assert set(np.unique(lv)) == {1, 2, 3}
    r = _pair(w, 24, usp.USP_FP64, sample_last=6)
    st = r["st"]
    gx, gy, gvx, gvy, gvz, ge, gl, gp = r["g"]
    assert len(gp) == st.n
    assert np.array_equal(gp, st.pid[:st.n])
    assert np.array_equal(gl, st.lev[:st.n])
    R = O.R(r["sp"])
    vth = math.sqrt(R * 200.0)
    assert np.max(np.abs(gx - st.x[:st.n])) < 1e-9
    assert np.max(np.abs(gy - st.y[:st.n])) < 1e-9
    for a, b in ((gvx, st.cx), (gvy, st.cy), (gvz, st.cz)):
        assert np.max(np.abs(a - b[:st.n])) < 1e-7 * vth
    assert np.max(np.abs(ge - st.erot[:st.n])) < 1e-7 * R * 200.0
    ncell = len(lv)
    assert len(r["gacc"]) == ncell * 12 + 2 + 4 * usp.USP_NSURF
    np.testing.assert_allclose(r["gacc"], r["acc"], rtol=1e-7, atol=1e-3)
    # every level holds particles, and the finest cells take part
    per_cell = r["acc"][:ncell * 12].reshape(ncell, 12)[:, 0]
    for L in (1, 2, 3):
        assert per_cell[lv == L].sum() > 1000
    for k in (usp.C_INFLOW, usp.C_OUTFLOW, usp.C_WALL_HITS, usp.C_CHOL_FIX, usp.C_NU_ZERO,
              usp.C_INTERP_FALLBACK):
        assert r["gcnt"][k] == r["cnt"][k], k
    assert r["gfl"] & usp.ERROR_FLAGS == 0


def test_fp64_refined_paper_grid_one_step_matches_oracle():
    """The paper's grid (640 x 480 level-1 cells, level 2 within 0.24 m, level
    3 within 0.155 m: 422,730 cells) at 10 particles per level-1 cell, one
    FP64 step from the initial state: every particle against the oracle."""
    w = I.cylinder_paper(ppc=10, refined=True)
    r = _pair(w, 1, usp.USP_FP64)
    st = r["st"]
    gx, gy, gvx, gvy, gvz, ge, gl, gp = r["g"]
    assert np.array_equal(gp, st.pid[:st.n])
    assert np.array_equal(gl, st.lev[:st.n])
    vth = math.sqrt(O.R(r["sp"]) * 200.0)
    assert np.max(np.abs(gvx - st.cx[:st.n])) < 1e-7 * vth
    assert np.max(np.abs(gx - st.x[:st.n])) < 1e-9
    for k in (usp.C_INFLOW, usp.C_OUTFLOW, usp.C_WALL_HITS):
        assert r["gcnt"][k] == r["cnt"][k], k


def test_fp32_refined_statistics_match_oracle():
    """FP32 GPU against the FP32-form oracle over 40 steps of the small
    refined case: per-level particle counts and mean translational
    temperatures agree within the sampling noise."""
    w = _small(ppc=48, seed=4)
    r = _pair(w, 40, usp.USP_FP32, sample_last=10)
    assert r["gfl"] & usp.ERROR_FLAGS == 0
    lv = usp.usp_plane_leaves(w.plane, arrays=True)[0]
    ncell = len(lv)
    R = O.R(r["sp"])
    for acc in (r["gacc"], r["acc"]):
        assert acc[ncell * 12] == 10
    ga = r["gacc"][:ncell * 12].reshape(ncell, 12)
    oa = r["acc"][:ncell * 12].reshape(ncell, 12)
    for L in (1, 2, 3):
        m = lv == L
        ng, no = ga[m, 0].sum(), oa[m, 0].sum()
        assert abs(ng - no) < 0.03 * no + 5 * math.sqrt(no)

        def temp(a):
            N = a[:, 0].sum()
            U = a[:, 1:4].sum(axis=0) / N
            return (a[:, 4:7].sum() / N - (U * U).sum()) / (3 * R)
        tg, to = temp(ga[m]), temp(oa[m])
        assert abs(tg - to) < 0.03 * to, (L, tg, to)


def test_fp32_refined_paper_grid_graph_run_invariants():
    """The paper's refined grid at 30 particles per level-1 cell (8.5M
    particles), FP32, 40 graph-replayed steps: exact bookkeeping, body empty,
    particles inside the domain and sorted by their cell (point location on
    the library's cell list), no error flag."""
    w = I.cylinder_paper(ppc=30, refined=True)
    sp, dto, dtg = _dts(w)
    x, y, cx, cy, cz, er, lev = _state(w, True)
    ctx = usp.usp_init_plane(w.species, w.plane, dtg, w.area_frac, x, y, cx, cy, cz, er, lev,
                             w.capacity, precision=usp.USP_FP32, seed=1)
    usp.usp_step(ctx, 40)
    fl, cnt = usp.usp_status(ctx)
    assert fl & usp.ERROR_FLAGS == 0
    n, nxt = usp.usp_plane_count(ctx)
    assert n == w.n_particles + cnt[usp.C_INFLOW] - cnt[usp.C_OUTFLOW]
    assert nxt == w.n_particles + cnt[usp.C_INFLOW]
    gx, gy, *_, gp = usp.usp_plane_get_particles(ctx)
    pl = w.plane
    assert np.all(gx * gx + gy * gy >= pl["cyl_r"] ** 2 * (1 - 1e-5))
    b = {k: float(np.float32(pl[k])) for k in ("x0", "x1", "y0", "y1")}
    assert np.all((gx >= b["x0"]) & (gx <= b["x1"]) & (gy >= b["y0"]) & (gy <= b["y1"]))
    cell = _leaf_of32(pl, gx, gy)
    assert np.mean(np.diff(cell) >= 0) > 1 - 1e-7
    assert len(np.unique(gp)) == n
