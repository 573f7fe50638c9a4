"""Pins of the oracle's refined plane grid (the three-level mesh of Sec. 5.C
and the reconstruction on non-uniform grids of Sec. 3.B): the leaf layout
against an independent enumeration and brute-force point location, the
reconstruction against bilinear fields it must reproduce exactly and against
the particle-number weighted average over a refined neighbour worked by hand,
and whole steps against invariants (a closed box conserves energy and keeps
every particle in its own leaf; rotational relaxation per step does not
depend on the level, which fixes the cell volumes)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I

KB = 1.380649e-23
DOM = dict(x0=-0.4, x1=0.4, y0=0.0, y1=0.6)


def _plane(nx=16, ny=12, levels=3, r2=0.3, r3=0.2, r=0.0, **kw):
    d = dict(nx=nx, ny=ny, cyl_xc=0.0, cyl_yc=0.0, cyl_r=r, amr_levels=levels, amr_r2=r2,
             amr_r3=r3, **DOM)
    d.update(kw)
    return O.plane(**d)


def _rects(pl):
    lv, ii, jj = O.plane_leaves(pl)
    s = 1.0 / (1 << (lv - 1)).astype(float)
    h = (pl.x1 - pl.x0) / pl.nx * s
    k = (pl.y1 - pl.y0) / pl.ny * s
    xl, yl = pl.x0 + ii * h, pl.y0 + jj * k
    return lv, xl, yl, h, k


# ---- layout ----------------------------------------------------------------
@pytest.mark.parametrize("levels,r2,r3,r", [(2, 0.3, 0.0, 0.0), (3, 0.3, 0.2, 0.0),
                                            (3, 0.3, 0.2, 0.1524), (1, 0.3, 0.2, 0.1)])
def test_leaf_layout_matches_independent_enumeration(levels, r2, r3, r):
    """The oracle's leaves equal the input module's enumeration (own code),
    tile the domain (areas add up; no overlap, checked on a point lattice),
    and the uniform grid is row-major level 1."""
    pl = _plane(levels=levels, r2=r2, r3=r3, r=r)
    lv, ii, jj = O.plane_leaves(pl)
    ref = I.refined_leaves(pl.nx, pl.ny, pl.x0, pl.x1, pl.y0, pl.y1, 0.0, 0.0, r, levels, r2, r3)
    for a, b in zip((lv, ii, jj), ref):
        np.testing.assert_array_equal(a, b)
    _, xl, yl, h, k = _rects(pl)
    area = (pl.x1 - pl.x0) * (pl.y1 - pl.y0)
    assert np.sum(h * k) == pytest.approx(area, rel=1e-12)
    # every lattice point (off the leaf edges) lies in exactly one leaf
    g = (np.arange(4 * 8 * pl.nx) + 0.5) / (4 * 8 * pl.nx)
    px = pl.x0 + g * (pl.x1 - pl.x0)
    py = pl.y0 + ((np.arange(4 * 8 * pl.ny) + 0.5) / (4 * 8 * pl.ny)) * (pl.y1 - pl.y0)
    X, Y = np.meshgrid(px[::7], py[::5])
    X, Y = X.ravel(), Y.ravel()
    inside = ((X[:, None] >= xl) & (X[:, None] < xl + h) & (Y[:, None] >= yl) & (Y[:, None] < yl + k))
    assert np.all(inside.sum(axis=1) == 1)
    if levels == 1:
        np.testing.assert_array_equal(lv, 1)
        np.testing.assert_array_equal(ii + pl.nx * jj, np.arange(pl.nx * pl.ny))


def test_refinement_follows_the_radii_and_the_body():
    """Level-2 leaves only inside r2 (+ a level-1 cell), level-3 only inside r3
    (+ a level-2 cell), no split cell lies wholly inside the body, and split
    cells come in complete 2 x 2 sets in (0,0), (1,0), (0,1), (1,1) order."""
    r = 0.1524
    pl = _plane(nx=32, ny=24, r2=0.3, r3=0.2, r=r)
    lv, xl, yl, h, k = _rects(pl)
    d = np.hypot(xl + h / 2, yl + k / 2)
    dx = (pl.x1 - pl.x0) / pl.nx
    assert np.all(d[lv == 2] < 0.3 + dx) and np.all(d[lv == 3] < 0.2 + dx)
    # a level-1 leaf centred within r2 lies wholly inside the body
    far = np.max([np.hypot(xl + a * h, yl + b * k) for a in (0, 1) for b in (0, 1)], axis=0)
    inner = (lv == 1) & (d < 0.3)
    assert inner.sum() > 10 and np.all(far[inner] <= r)
    # a leaf at level >= 2 lies within one level-1 cell of the body's outside
    assert np.all(far[lv >= 2] > r - 2 * dx)
    # level-3 leaves come in 2 x 2 sets in the order (0,0), (1,0), (0,1), (1,1)
    _, ii, jj = O.plane_leaves(pl)
    idx = np.nonzero(lv == 3)[0]
    first = idx[(ii[idx] % 2 == 0) & (jj[idx] % 2 == 0)]
    assert len(first) * 4 == len(idx)
    for q, (a, b) in enumerate([(0, 0), (1, 0), (0, 1), (1, 1)]):
        assert np.all(lv[first + q] == 3)
        assert np.all(ii[first + q] == ii[first] + a) and np.all(jj[first + q] == jj[first] + b)
    # the leaves of each level-1 cell fill it and are numbered together, in
    # row-major order of the level-1 cells
    parent = (jj >> (lv - 1)) * pl.nx + (ii >> (lv - 1))
    assert np.all(np.diff(parent) >= 0)
    area = np.bincount(parent, weights=h * k, minlength=pl.nx * pl.ny)
    np.testing.assert_allclose(area, dx * (pl.y1 - pl.y0) / pl.ny, rtol=1e-12)


def test_leaf_of_is_brute_force_containment():
    pl = _plane(nx=16, ny=12, r=0.1)
    _, xl, yl, h, k = _rects(pl)
    rng = np.random.default_rng(4)
    for _ in range(3000):
        x = rng.uniform(pl.x0, pl.x1)
        y = rng.uniform(pl.y0, pl.y1)
        l = O.plane_leaf_of(pl, x, y)
        assert xl[l] <= x < xl[l] + h[l] and yl[l] <= y < yl[l] + k[l]


def test_neighbouring_levels_may_differ_by_one_only():
    """Level 3 reaching to the level-2 boundary leaves level-1 leaves beside
    level-3 ones: the grid is rejected (count -1, the step refuses it)."""
    assert O.plane_nleaf(_plane(r2=0.2, r3=0.2)) == -1
    assert O.plane_nleaf(_plane(r2=0.3, r3=0.2)) > 0


# ---- reconstruction -------------------------------------------------------------
def _bilinear(x, y, cross=1.0):
    f = np.empty(O.NFIELD)
    for q in range(O.NFIELD):
        a, b, c, d = 1.0 + q, 0.3 - 0.05 * q, -0.7 + 0.1 * q, 0.25 * (q % 3 - 1) * cross
        f[q] = a + b * x + c * y + d * x * y
    return f


@pytest.mark.parametrize("r", [0.0, 0.1524])
def test_bilinear_field_is_reproduced_across_levels(r):
    """With cell averages of a bilinear field (its value at the leaf centre)
    and equal particle counts, the reconstruction at any point of a whole leaf
    returns the field exactly: same-level neighbours, the mean of four finer
    leaves (centre of their quarters), the coarser leaf's own polynomial at the
    square's centre, and the one-sided fallbacks at the domain edge all agree
    with a bilinear polynomial.  Beside the body a cut diagonal drops the cross
    term, so there the field is linear."""
    cross = 1.0 if r == 0.0 else 0.0
    pl = _plane(nx=16, ny=12, r=r)
    lv, xl, yl, h, k = _rects(pl)
    n = len(lv)
    af = np.ones(n)
    if r > 0:
        af = I.refined_cut_fractions(pl.nx, pl.ny, pl.x0, pl.x1, pl.y0, pl.y1, 0.0, 0.0, r,
                                     O.plane_leaves(pl))
    F = np.array([_bilinear(xl[l] + h[l] / 2, yl[l] + k[l] / 2, cross) for l in range(n)])
    counts = np.full(n, 6, dtype=np.int64)
    rng = np.random.default_rng(8)
    for l in rng.permutation(n)[:600]:
        if af[l] < 1.0:
            continue
        x = xl[l] + rng.uniform(0.02, 0.98) * h[l]
        y = yl[l] + rng.uniform(0.02, 0.98) * k[l]
        out = O.plane_reconstruct(pl, counts, af, F, int(l), x, y)
        np.testing.assert_allclose(out, _bilinear(x, y, cross), rtol=1e-12, atol=1e-12)


def test_refined_neighbour_is_the_count_weighted_average():
    """A level-1 leaf whose +x neighbour square is split into four level-2
    leaves, every other neighbour unusable: at (x_c + delta, y_c) the value is
    F + (P - F) delta / dx with P = sum N_q F_q / sum N_q, worked by hand."""
    pl = _plane(nx=16, ny=12, levels=2, r2=0.3, r3=0.0)
    lv, xl, yl, h, k = _rects(pl)
    dx = (pl.x1 - pl.x0) / pl.nx
    # a level-1 leaf with a split cell on its right
    t = None
    for l in np.nonzero(lv == 1)[0]:
        q = O.plane_leaf_of(pl, xl[l] + 1.25 * dx, yl[l] + 0.25 * k[l])
        if lv[q] == 2 and xl[l] > pl.x0 + dx and yl[l] > pl.y0 + k[l]:
            t = l
            break
    assert t is not None
    n = len(lv)
    af = np.full(n, 0.5)            # unusable neighbours everywhere ...
    counts = np.full(n, 4, dtype=np.int64)
    quarters = [O.plane_leaf_of(pl, xl[t] + dx * (1.25 + 0.5 * a), yl[t] + k[t] * (0.25 + 0.5 * b))
                for b in (0, 1) for a in (0, 1)]
    af[t] = 1.0
    af[quarters] = 1.0              # ... but the four finer leaves on the right
    Nq = np.array([2, 3, 5, 7])
    counts[quarters] = Nq
    F = np.zeros((n, O.NFIELD))
    F[t] = 10.0
    Fq = np.array([[20.0 + a + 0.1 * f for f in range(O.NFIELD)] for a in (1.0, 5.0, -2.0, 3.0)])
    F[quarters] = Fq
    P = (Nq[:, None] * Fq).sum(axis=0) / Nq.sum()
    xc, yc = xl[t] + 0.5 * dx, yl[t] + 0.5 * k[t]
    for delta in (0.1 * dx, 0.45 * dx):
        out = O.plane_reconstruct(pl, counts, af, F, int(t), xc + delta, yc + 0.2 * k[t])
        np.testing.assert_allclose(out, F[t] + (P - F[t]) * delta / dx, rtol=1e-13)
    # left half: the right square replaces the unusable left one (one-sided)
    out = O.plane_reconstruct(pl, counts, af, F, int(t), xc - 0.3 * dx, yc)
    np.testing.assert_allclose(out, F[t] + (P - F[t]) * (-0.3), rtol=1e-13)
    # a finer cell with a single particle has no stress or temperature: the
    # square is unusable and the x slope vanishes
    counts[quarters[2]] = 1
    out = O.plane_reconstruct(pl, counts, af, F, int(t), xc + 0.3 * dx, yc)
    np.testing.assert_allclose(out, F[t], rtol=1e-13)


# ---- whole steps -------------------------------------------------------------
def _box(ppc=320, T_tr=200.0, T_rot=200.0, seed=3):
    w = I.cylinder_flow(nx=12, ny=8, ppc=ppc, U_inf=0.0, T_inf=T_tr, cylinder=False,
                        amr_levels=3, amr_r2=0.26, amr_r3=0.08, seed=seed)
    w.plane["bc"] = (O.BC_SPECULAR,) * 4
    w.plane["inflow"] = (0, 0, 0, 0)
    rng = np.random.default_rng(seed)
    p = I.equilibrium_particles(rng, w.n_particles, w.species["m"], w.species["theta_v"],
                                T_tr=T_tr, T_rot=T_rot, T_vib=T_tr)
    return w, p


def test_closed_refined_box_conserves_energy_and_sorts_into_leaves():
    w, p = _box(ppc=80)
    sp = O.species(**w.species)
    pl = O.plane(**w.plane)
    dt = 0.5 * O.tau_c(sp, w.plane["n_inf"], 200.0)
    st = O.PlaneState(w.x, w.y, p.cx, p.cy, p.cz, p.erot, p.lev, w.capacity)
    R = KB / w.species["m"]

    def energy():
        x, y, cx, cy, cz, er, lev, _ = st.live()
        return np.sum(0.5 * (cx * cx + cy * cy + cz * cz) + er + R * sp.theta_v * lev)
    E0, N0 = energy(), st.n
    off, fl, cnt = O.plane_step(sp, 0, 11, 0, 6, pl, w.area_frac, dt, st)
    assert fl & (O.F_A_NONPOS | O.F_CAPACITY) == 0
    assert st.n == N0 and len(np.unique(st.pid[:st.n])) == N0
    assert energy() == pytest.approx(E0, rel=1e-11)
    lv, xl, yl, h, k = _rects(pl)
    cell = np.repeat(np.arange(len(lv)), np.diff(off))
    x, y = st.x[:st.n], st.y[:st.n]
    assert np.all((x >= xl[cell]) & (x <= xl[cell] + h[cell]) &
                  (y >= yl[cell]) & (y <= yl[cell] + k[cell]))


def test_relaxation_per_step_does_not_depend_on_the_level():
    """Rotational non-equilibrium in a closed box of uniform density: the
    post-step rotational temperature of every cell is its target, whose
    distance from T_tr shrinks by a factor fixed by the density (the cell's
    particle count over its volume, area / 4^(level-1)).  The mean factor
    agrees between levels; a volume off by 4 would move it by about 0.1."""
    w, p = _box(ppc=320, T_rot=80.0)
    sp = O.species(**w.species)
    pl = O.plane(**w.plane)
    dt = 0.5 * O.tau_c(sp, w.plane["n_inf"], 200.0)
    st = O.PlaneState(w.x, w.y, p.cx, p.cy, p.cz, p.erot, p.lev, w.capacity)
    R = KB / w.species["m"]
    lv = O.plane_leaves(pl)[0]
    x0, y0 = st.x[:st.n].copy(), st.y[:st.n].copy()
    c0 = np.array([O.plane_leaf_of(pl, a, b) for a, b in zip(x0, y0)])
    before = np.bincount(c0, weights=st.erot[:st.n], minlength=len(lv)) / np.maximum(
        np.bincount(c0, minlength=len(lv)), 1) / R
    off, fl, _ = O.plane_step(sp, 0, 13, 0, 1, pl, w.area_frac, dt, st)
    assert fl & O.F_A_NONPOS == 0
    cnt = np.diff(off)
    after = np.add.reduceat(st.erot[:st.n], off[:-1].clip(max=st.n - 1)) / np.maximum(cnt, 1) / R
    ok = cnt >= 8
    ratio = (200.0 - after) / (200.0 - before)
    r1 = np.median(ratio[ok & (lv == 1)])
    for L in (2, 3):
        m = ok & (lv == L)
        assert m.sum() >= 10
        assert abs(np.median(ratio[m]) - r1) < 0.03, (L, np.median(ratio[m]), r1)
    assert 0.05 < 1.0 - r1 < 0.95
