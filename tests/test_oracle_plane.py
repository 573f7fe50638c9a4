"""Pins of the oracle's 2D plane path (the cylinder set-up of Sec. 5.C): the
freestream inflow against kinetic theory, the 2D reconstruction of Sec. 3.B
against exactly representable fields, and whole steps against invariants
(uniform stream stays uniform, a closed specular box conserves energy, the
cylinder stays empty, particle bookkeeping)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I

KB = 1.380649e-23


def _R(sp):
    return KB / sp["m"]


# ---- inflow -----------------------------------------------------------------
@pytest.mark.parametrize("s", [0.0, 0.4, -0.7, 2.0, 8.37])
def test_inflow_flux_is_the_half_range_integral(s):
    """One-way flux n <v_n; v_n > 0> of a drifting Maxwellian by quadrature."""
    integrate = pytest.importorskip("scipy.integrate")
    RT = 296.8 * 200.0
    u = s * math.sqrt(2 * RT)
    n = 1.2e21
    f = lambda v: v * math.exp(-(v - u) ** 2 / (2 * RT)) / math.sqrt(2 * math.pi * RT)
    ref = n * integrate.quad(f, 0.0, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]
    assert O.inflow_flux(n, RT, u) == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("s", [0.0, 0.4, -0.7, 8.37])
def test_inflow_normal_speed_is_flux_weighted(s):
    """Entering normal speeds have density proportional to v exp(-(v-u)^2/2RT)
    on v > 0: Kolmogorov-Smirnov against the numerically integrated CDF, and
    the mean against the ratio of the two half-range moments."""
    stats = pytest.importorskip("scipy.stats")
    integrate = pytest.importorskip("scipy.integrate")
    RT = 296.8 * 200.0
    sc = math.sqrt(2 * RT)
    u = s * sc
    M = 40000
    v = np.array([O.inflow_normal_speed(RT, u, pid, 7, 99)[0] for pid in range(M)]) / sc
    assert np.all(v > 0)
    dens = lambda w: w * math.exp(-(w - s) ** 2)
    lo, hi = max(0.0, s - 9.0), s + 9.0
    Z = integrate.quad(dens, lo, hi, epsabs=0, epsrel=1e-12)[0]
    grid = np.linspace(lo, hi, 4001)
    pdf = np.array([dens(w) for w in grid]) / Z
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(grid))])
    F = lambda x: np.interp(x, grid, cdf)
    assert stats.kstest(v, F).pvalue > 1e-3
    m1 = integrate.quad(lambda w: w * dens(w), lo, hi, epsabs=0, epsrel=1e-12)[0] / Z
    m2 = integrate.quad(lambda w: w * w * dens(w), lo, hi, epsabs=0, epsrel=1e-12)[0] / Z
    assert v.mean() == pytest.approx(m1, abs=5 * math.sqrt((m2 - m1 * m1) / M))


# ---- 2D reconstruction ------------------------------------------------------
def _grid(nx=8, ny=6):
    pl = O.plane(nx=nx, ny=ny, x0=-1.0, x1=1.0, y0=0.0, y1=1.5, cyl_r=0.0, T_wall=300.0,
                 n_inf=1e20, T_inf=300.0, U_inf=0.0, bc=(0, 0, 1, 0), inflow=(0, 0, 0, 0),
                 F_num=1.0, depth=1.0, reconstruct=1)
    dx, dy = 2.0 / nx, 1.5 / ny
    xc = -1.0 + (np.arange(nx) + 0.5) * dx
    yc = 0.0 + (np.arange(ny) + 0.5) * dy
    return pl, dx, dy, xc, yc


def _fields(fun, xc, yc):
    nx, ny = len(xc), len(yc)
    F = np.zeros((ny * nx, O.NFIELD))
    for j in range(ny):
        for i in range(nx):
            F[j * nx + i] = [fun(xc[i], yc[j], k) for k in range(O.NFIELD)]
    return F


def _lin(x, y, k):
    return 3.0 + k + (0.5 + 0.1 * k) * x - (1.3 - 0.2 * k) * y


def _bilin(x, y, k):
    return _lin(x, y, k) + (0.7 + 0.05 * k) * x * y


def test_reconstruction_reproduces_linear_fields_everywhere():
    """A linear field is exact in every cell with a usable neighbour in each
    direction, whichever side the stencil takes (domain edge, cut or sparse
    neighbour -> the opposite side); the cross term vanishes on it."""
    pl, dx, dy, xc, yc = _grid()
    nx, ny = pl.nx, pl.ny
    counts = np.full(nx * ny, 5, dtype=np.int64)
    af = np.ones(nx * ny)
    af[2 * nx + 3] = 0.4          # a cut cell: never a neighbour
    counts[4 * nx + 5] = 1        # a sparse cell: never a neighbour
    F = _fields(_lin, xc, yc)
    usable = lambda i, j: 0 <= i < nx and 0 <= j < ny and af[j * nx + i] >= 1 and \
        counts[j * nx + i] >= 2
    rng = np.random.default_rng(3)
    for cell in range(nx * ny):
        i, j = cell % nx, cell // nx
        for _ in range(6):
            x = xc[i] + rng.uniform(-0.5, 0.5) * dx
            y = yc[j] + rng.uniform(-0.5, 0.5) * dy
            out = O.plane_reconstruct(pl, counts, af, F, cell, x, y)
            # a direction without any usable neighbour has no slope
            xe = x if (usable(i - 1, j) or usable(i + 1, j)) else xc[i]
            ye = y if (usable(i, j - 1) or usable(i, j + 1)) else yc[j]
            ref = [_lin(xe, ye, k) for k in range(O.NFIELD)]
            np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_reconstruction_reproduces_bilinear_fields_with_full_quadrant():
    """A bilinear field is exact where the quadrant's x, y and diagonal
    neighbours are all usable (interior cells)."""
    pl, dx, dy, xc, yc = _grid()
    nx, ny = pl.nx, pl.ny
    counts = np.full(nx * ny, 5, dtype=np.int64)
    af = np.ones(nx * ny)
    F = _fields(_bilin, xc, yc)
    rng = np.random.default_rng(4)
    for j in range(ny):
        for i in range(nx):
            cell = j * nx + i
            for _ in range(6):
                x = xc[i] + rng.uniform(-0.5, 0.5) * dx
                y = yc[j] + rng.uniform(-0.5, 0.5) * dy
                out = O.plane_reconstruct(pl, counts, af, F, cell, x, y)
                ref = [_bilin(x, y, k) for k in range(O.NFIELD)]
                np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_reconstruction_uses_the_particles_quadrant():
    """A field with a kink at one cell's centroid: on each side the
    reconstruction follows that side's neighbour, so the quadrant choice (and
    its tie at the centroid going to +) is visible."""
    pl, dx, dy, xc, yc = _grid()
    nx, ny = pl.nx, pl.ny
    counts = np.full(nx * ny, 5, dtype=np.int64)
    af = np.ones(nx * ny)
    i0, j0 = 4, 3
    kink = lambda x, y, k: abs(x - xc[i0]) * (1 + k) + 2.0 * abs(y - yc[j0])
    F = _fields(kink, xc, yc)
    cell = j0 * nx + i0
    for sx in (-1, 1):
        for sy in (-1, 1):
            x = xc[i0] + sx * 0.3 * dx
            y = yc[j0] + sy * 0.2 * dy
            out = O.plane_reconstruct(pl, counts, af, F, cell, x, y)
            ref = [kink(x, y, k) for k in range(O.NFIELD)]
            np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)
    out = O.plane_reconstruct(pl, counts, af, F, cell, xc[i0], yc[j0])
    np.testing.assert_allclose(out, F[cell], rtol=0, atol=1e-12)


def test_reconstruction_without_neighbours_keeps_the_cell_value():
    pl, dx, dy, xc, yc = _grid(nx=3, ny=3)
    counts = np.zeros(9, dtype=np.int64)
    counts[4] = 7
    af = np.ones(9)
    F = _fields(_bilin, xc, yc)
    out = O.plane_reconstruct(pl, counts, af, F, 4, xc[1] + 0.2 * dx, yc[1] - 0.4 * dy)
    np.testing.assert_array_equal(out, F[4])


# ---- whole steps --------------------------------------------------------------
def _run(w, steps, seed=5, form=0):
    sp = O.species(**w.species)
    pl = O.plane(**w.plane)
    dt = w.dt_over_tau_c * O.tau_c(sp, w.plane["n_inf"], w.plane["T_inf"])
    p = w.particles
    st = O.PlaneState(w.x, w.y, p.cx, p.cy, p.cz, p.erot, p.lev, w.capacity)
    off, fl, cnt = O.plane_step(sp, form, seed, 0, steps, pl, w.area_frac, dt, st)
    return sp, pl, dt, st, off, fl, cnt


@pytest.mark.parametrize("U", [0.0, 2883.3])
def test_uniform_stream_stays_uniform(U):
    """Equilibrium freestream through an empty domain with inflow on every
    open side: the injected flux, speed distribution and entry times keep the
    density uniform up to the inflow faces and the bulk state unchanged."""
    w = I.cylinder_flow(nx=16, ny=10, ppc=80, U_inf=U, cylinder=False)
    w.plane["inflow"] = (1, 1, 0, 1)
    N0 = w.n_particles
    steps = 30
    sp, pl, dt, st, off, fl, cnt = _run(w, steps)
    assert fl & (O.F_CHOL_FAIL_AFTER_FIX | O.F_A_NONPOS | O.F_CAPACITY) == 0
    assert st.n == N0 + cnt[O.C_INFLOW] - cnt[O.C_OUTFLOW]
    assert abs(st.n - N0) < 4 * math.sqrt(N0)
    nx, ny = pl.nx, pl.ny
    counts = np.diff(off).reshape(ny, nx)
    col = counts.sum(axis=0).astype(float)
    mean, sig = col.mean(), math.sqrt(col.mean())
    # boundary columns (where inflow enters) hold the same density
    assert abs(col[0] - mean) < 5 * sig and abs(col[-1] - mean) < 5 * sig
    row = counts.sum(axis=1).astype(float)
    assert abs(row[-1] - row.mean()) < 5 * math.sqrt(row.mean())
    x, y, cx, cy, cz, er, lev, pid = st.live()
    R = _R(w.species)
    assert cx.mean() == pytest.approx(U, abs=5 * math.sqrt(R * 200.0 / st.n))
    Ttr = (cx.var() + cy.var() + cz.var()) / (3 * R)
    assert Ttr == pytest.approx(200.0, rel=0.02)
    assert er.mean() / R == pytest.approx(200.0, rel=0.03)
    assert len(np.unique(pid)) == st.n


def test_closed_specular_box_conserves_energy_and_particles():
    """All sides specular, no body, no inflow: every collision step conserves
    each cell's momentum and energy (Sec. 4.C) and the walls conserve energy,
    so the total energy and the particle count are invariant."""
    w = I.cylinder_flow(nx=12, ny=8, ppc=40, U_inf=900.0, cylinder=False)
    w.plane["bc"] = (O.BC_SPECULAR,) * 4
    w.plane["inflow"] = (0, 0, 0, 0)
    sp = O.species(**w.species)
    R = O.R(sp)
    p = w.particles

    def energy(cx, cy, cz, er, lev):
        return np.sum(0.5 * (cx * cx + cy * cy + cz * cz) + er + lev * R * sp.theta_v)

    E0 = energy(p.cx, p.cy, p.cz, p.erot, p.lev)
    _, pl, dt, st, off, fl, cnt = _run(w, 25)
    assert st.n == w.n_particles
    assert cnt[O.C_INFLOW] == 0 and cnt[O.C_OUTFLOW] == 0 and cnt[O.C_WALL_HITS] > 0
    x, y, cx, cy, cz, er, lev, pid = st.live()
    assert energy(cx, cy, cz, er, lev) == pytest.approx(E0, rel=1e-11)
    assert np.all((x >= pl.x0) & (x <= pl.x1) & (y >= pl.y0) & (y <= pl.y1))


def test_cylinder_run_keeps_the_body_empty_and_books_every_particle():
    w = I.cylinder_flow(nx=48, ny=32, ppc=10)
    N0 = w.n_particles
    sp, pl, dt, st, off, fl, cnt = _run(w, 40)
    assert fl & (O.F_CHOL_FAIL_AFTER_FIX | O.F_A_NONPOS | O.F_CAPACITY | O.F_WALL_CAP) == 0
    assert cnt[O.C_WALL_HITS] > 0 and cnt[O.C_INFLOW] > 0 and cnt[O.C_OUTFLOW] > 0
    assert st.n == N0 + cnt[O.C_INFLOW] - cnt[O.C_OUTFLOW]
    x, y, cx, cy, cz, er, lev, pid = st.live()
    r = w.plane["cyl_r"]
    assert np.all(x * x + y * y >= r * r * (1 - 1e-9))
    assert np.all((y >= pl.y0) & (y <= pl.y1) & (x >= pl.x0) & (x <= pl.x1))
    assert len(np.unique(pid)) == st.n
    assert st.next_pid == N0 + cnt[O.C_INFLOW]
    # sorted by cell, offsets consistent with positions
    cell = np.clip(np.floor((x - pl.x0) / ((pl.x1 - pl.x0) / pl.nx)).astype(int), 0, pl.nx - 1) + \
        pl.nx * np.clip(np.floor((y - pl.y0) / ((pl.y1 - pl.y0) / pl.ny)).astype(int), 0, pl.ny - 1)
    assert np.all(np.diff(cell) >= 0)
    np.testing.assert_array_equal(np.searchsorted(cell, np.arange(pl.nx * pl.ny + 1)), off)
    # a bow shock forms: density ahead of the body exceeds the freestream
    ny, nx = pl.ny, pl.nx
    counts = np.diff(off).reshape(ny, nx)
    xs = pl.x0 + (np.arange(nx) + 0.5) * (pl.x1 - pl.x0) / nx
    ahead = (xs > -r - 0.05) & (xs < -r)
    assert counts[0, ahead].mean() > 1.5 * 10


def test_reconstructed_temperature_is_the_trace_of_reconstructed_stress():
    """T_tr = tr(Pi)/3R holds at every particle position when it holds for the
    cell averages: the reconstruction of Sec. 3.B is linear in the cell values."""
    pl, dx, dy, xc, yc = _grid()
    nx, ny = pl.nx, pl.ny
    R = 296.9
    rng = np.random.default_rng(9)
    F = rng.uniform(1.0, 2.0, (nx * ny, O.NFIELD)) * 1e4
    F[:, 3] = (F[:, 6] + F[:, 7] + F[:, 8]) / (3 * R)
    counts = np.full(nx * ny, 5, dtype=np.int64)
    counts[rng.integers(0, nx * ny, 6)] = 1
    af = np.ones(nx * ny)
    af[rng.integers(0, nx * ny, 4)] = 0.5
    for cell in range(nx * ny):
        i, j = cell % nx, cell // nx
        x = xc[i] + rng.uniform(-0.5, 0.5) * dx
        y = yc[j] + rng.uniform(-0.5, 0.5) * dy
        f = O.plane_reconstruct(pl, counts, af, F, cell, x, y)
        assert f[3] == pytest.approx((f[6] + f[7] + f[8]) / (3 * R), rel=1e-12)


def test_surface_tallies_of_a_gas_at_rest_at_the_wall_temperature():
    """Cylinder in a closed specular box of N2 at rest at T = T_wall: the
    surface tallies give the ideal-gas pressure n k_B T on the wall (half from
    the incoming, half from the re-emitted momentum flux), and no net shear
    and no net heat flux (the re-emitted gas carries back what arrives).
    About 3,000 wall events: bars of three standard deviations."""
    T = 500.0
    w = I.cylinder_flow(nx=24, ny=16, ppc=200, U_inf=0.0, T_inf=T)
    w.plane["bc"] = (O.BC_SPECULAR,) * 4
    w.plane["inflow"] = (0, 0, 0, 0)
    sp = O.species(**w.species)
    pl = O.plane(**w.plane)
    dt = 1.0 * O.tau_c(sp, w.plane["n_inf"], T)
    p = w.particles
    st = O.PlaneState(w.x, w.y, p.cx, p.cy, p.cz, p.erot, p.lev, w.capacity)
    acc = O.plane_acc(pl)
    steps = 150
    fl, _ = O.plane_step(sp, 0, 5, 0, steps, pl, w.area_frac, dt, st, acc)[1:]
    assert fl & (O.F_A_NONPOS | O.F_CAPACITY) == 0
    ncell = pl.nx * pl.ny
    assert acc[ncell * O.NACC] == steps
    s = acc[ncell * O.NACC + 2:].reshape(-1, 4)
    nb = len(s)
    phi = -math.pi + (np.arange(nb) + 0.5) * 2 * math.pi / nb
    up = phi > 0.05
    assert np.all(s[phi < -0.05, 3] == 0)          # no wall below the symmetry plane
    assert s[:, 3].sum() > 2000
    m = sp.m
    area = w.plane["cyl_r"] * (2 * math.pi / nb) * w.plane["depth"]
    fx = w.plane["F_num"] * m * s[:, 0] / (steps * dt)
    fy = w.plane["F_num"] * m * s[:, 1] / (steps * dt)
    press = -(fx * np.cos(phi) + fy * np.sin(phi)) / area
    shear = (fx * np.sin(phi) - fy * np.cos(phi)) / area
    p_ideal = w.plane["n_inf"] * KB * T
    assert np.mean(press[up]) == pytest.approx(p_ideal, rel=0.06)
    assert abs(np.mean(shear[up])) < 0.06 * p_ideal
    # heat flux: energy in minus out, against the one-way energy flux scale
    q = w.plane["F_num"] * m * s[:, 2] / (steps * dt) / area
    one_way = p_ideal * math.sqrt(8 * O.R(sp) * T / math.pi)
    assert abs(np.mean(q[up])) < 0.08 * one_way


# ---- the plain FPM method on the plane (Sec. 2.B-C, cell values) ------------
@pytest.mark.parametrize("form", [0, 1])
def test_plane_fpm_step_is_the_homogeneous_fpm_step_in_one_cell(form):
    """One 1 m x 1 m cell with specular sides and particles far from them (no
    wall event in the step): the plane step with the plain FPM method is the
    homogeneous FPM step (pinned by its own closed forms) at the cell's density
    n = N F_num / V, particle for particle, bitwise."""
    rng = np.random.default_rng(21)
    w = I.cylinder_flow(nx=1, ny=1, ppc=1, cylinder=False)
    N = 3000
    sp_d = w.species
    p = I.equilibrium_particles(rng, N, sp_d["m"], sp_d["theta_v"], U=(40.0, -10.0, 5.0),
                                T_tr=3000.0, T_rot=800.0, T_vib=1500.0)
    pl_d = dict(w.plane, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=(O.BC_SPECULAR,) * 4,
                inflow=(0, 0, 0, 0), method=1, reconstruct=1)
    pl_d["F_num"] = 1e23 / N
    x = rng.uniform(0.45, 0.55, N)
    y = rng.uniform(0.45, 0.55, N)
    sp = O.species(**sp_d)
    pl = O.plane(**pl_d)
    dt = 0.7 * O.tau_c(sp, 1e23, 3000.0)
    st = O.PlaneState(x, y, p.cx, p.cy, p.cz, p.erot, p.lev, N + 16)
    _, fl, cnt = O.plane_step(sp, form, 9, 4, 1, pl, np.ones(1), dt, st)
    assert cnt[O.C_WALL_HITS] == 0 and st.n == N
    hs = O.State.from_arrays(p.cx, p.cy, p.cz, p.erot, p.lev)
    O.homog_step_fpm(sp, form, 9, 4, 1, np.array([0, N]), np.array([1e23]), np.array([dt]), hs)
    for a, b in ((st.cx, hs.cx), (st.cy, hs.cy), (st.cz, hs.cz), (st.erot, hs.erot)):
        np.testing.assert_array_equal(a[:N], b)
    np.testing.assert_array_equal(st.lev[:N], hs.lev)
    # and it differs from the USP-FPM step of the same cell
    pl2 = O.plane(**dict(pl_d, method=0))
    st2 = O.PlaneState(x, y, p.cx, p.cy, p.cz, p.erot, p.lev, N + 16)
    O.plane_step(sp, form, 9, 4, 1, pl2, np.ones(1), dt, st2)
    assert not np.array_equal(st2.cx[:N], hs.cx)
