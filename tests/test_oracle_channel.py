"""Pins of the oracle's 1D channel (spatial) path: diffuse-wall law, the
first-order reconstruction of Sec. 3.B, exact momentum bookkeeping, closed-box
equilibrium and the developed force-driven Poiseuille profile (Sec. 5.B)."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I

KB = 1.380649e-23


def _setup(w, **over):
    sp = O.species(**w.species)
    chd = dict(w.channel)
    chd.update(over)
    ch = O.channel(**chd)
    dt = w.dt_over_tau_c * O.tau_c(sp, w.n, w.channel["T_wall"])
    p = w.particles
    st = O.ChannelState.from_arrays(w.y, p.cx, p.cy, p.cz, p.erot, p.lev)
    return sp, ch, dt, st


def test_diffuse_wall_law():
    """Fully diffuse wall at T_w: flux-weighted half-range Maxwellian normal
    speed (Rayleigh, variance R T_w), Maxwellian tangential components,
    exponential eps_rot (mean R T_w), geometric levels at T_w; the normal
    velocity points into the gas."""
    sp = O.species(**I.n2_vss_species())
    R = O.R(sp)
    Tw = 2500.0
    n = 20000
    out = np.array([O.wall_reemit(sp, 0, 3, pid, 7, 0, Tw, pid % 2 == 0)[0] for pid in range(n)])
    lev = np.array([O.wall_reemit(sp, 0, 3, pid, 7, 0, Tw, True)[1] for pid in range(n)])
    s = math.sqrt(R * Tw)
    cy = out[:, 1]
    up = np.arange(n) % 2 == 0
    assert np.all(cy[up] > 0) and np.all(cy[~up] < 0)
    assert stats.kstest(np.abs(cy) / s, "rayleigh").pvalue > 1e-3
    assert stats.kstest(out[:, 0] / s, "norm").pvalue > 1e-3
    assert stats.kstest(out[:, 2] / s, "norm").pvalue > 1e-3
    assert stats.kstest(out[:, 3] / (R * Tw), "expon").pvalue > 1e-3
    q = math.exp(-sp.theta_v / Tw)
    kmax = 5
    obs = np.array([(lev == k).sum() for k in range(kmax)] + [(lev >= kmax).sum()])
    pm = np.array([(1 - q) * q ** k for k in range(kmax)] + [q ** kmax])
    assert stats.chisquare(obs, n * pm).pvalue > 1e-3


def test_reconstruction_reproduces_linear_fields():
    """A field linear in y is reproduced exactly everywhere, including the
    wall cells (stencil from the opposite side) and next to a cell holding
    too few particles; a quadratic field is matched at the centroids."""
    ny, L = 10, 1e-4
    ch = O.channel(ny=ny, L=L, T_wall=300.0, g=0.0, F_num=1.0, area=1.0, reconstruct=1)
    dy = L / ny
    yc = (np.arange(ny) + 0.5) * dy
    rng = np.random.default_rng(4)
    a = rng.uniform(100, 200, 13)
    b = rng.uniform(-1e6, 1e6, 13)
    F = (a[None, :] + b[None, :] * yc[:, None])
    for counts in (np.full(ny, 50), np.array([50, 50, 50, 1, 50, 50, 0, 50, 50, 50])):
        for c in range(ny):
            if counts[c] < 2:
                continue
            for y in rng.uniform(c * dy, (c + 1) * dy, 5).tolist() + [c * dy, (c + 1) * dy, yc[c]]:
                out = O.channel_reconstruct(ch, counts, F, c, y)
                assert np.allclose(out, a + b * y, rtol=1e-12, atol=1e-9)
    Fq = (1e9 * (yc - 0.4 * L) ** 2)[:, None] * np.ones(13)
    for c in range(ny):
        assert np.allclose(O.channel_reconstruct(ch, np.full(ny, 50), Fq, c, yc[c]), Fq[c])


def test_momentum_bookkeeping_is_exact():
    """Collisions conserve momentum per cell (Sec. 4.C), so the gas x-momentum
    changes only by the body force and by what the walls take."""
    w = I.channel_poiseuille(ny=16, ppc=60, steps=0)
    sp, ch, dt, st = _setup(w)
    acc = np.zeros(ch.ny * O.NACC + 2)
    p0 = st.cx.sum()
    steps = 40
    off, fl, cnt = O.channel_step(sp, 0, 5, 0, steps, ch, dt, st, acc)
    assert fl == 0 and cnt[O.C_WALL_HITS] > 0
    n = len(st.y)
    expected = p0 + n * ch.g * dt * steps - acc[ch.ny * O.NACC + 1]
    assert st.cx.sum() == pytest.approx(expected, rel=1e-11, abs=1e-9 * n)
    assert np.all(np.diff(off) >= 0) and off[-1] == n
    assert np.all((st.y >= 0) & (st.y <= ch.L))


def test_closed_box_keeps_wall_equilibrium():
    """No force, gas at the wall temperature: it stays at T_w, at rest.  One
    run's mean temperature over the box scatters by 1.4 % between seeds (16
    cells of 100 particles, 100 averaged steps), so eight seeds are pooled."""
    w = I.channel_poiseuille(ny=16, ppc=100, g=0.0, steps=0)
    acc = None
    for seed in range(1, 9):
        sp, ch, dt, st = _setup(w)
        a1 = np.zeros(ch.ny * O.NACC + 2)
        O.channel_step(sp, 0, seed, 0, 100, ch, dt, st)
        O.channel_step(sp, 0, seed, 100, 100, ch, dt, st, a1)
        acc = a1 if acc is None else acc + a1
    R = O.R(sp)
    a = acc[: ch.ny * O.NACC].reshape(ch.ny, O.NACC)
    N = a[:, 0]
    U = a[:, 1:4] / N[:, None]
    T = ((a[:, 4] + a[:, 5] + a[:, 6]) / N - (U ** 2).sum(1)) / (3 * R)
    Trot = a[:, 10] / N / R
    # 100 particles per cell: per-cell statistical scatter of a few percent
    assert abs(T.mean() / 300.0 - 1) < 0.015 and np.all(np.abs(T / 300.0 - 1) < 0.08)
    assert abs(Trot.mean() / 300.0 - 1) < 0.015 and np.all(np.abs(Trot / 300.0 - 1) < 0.08)
    vth = math.sqrt(R * 300)
    assert abs(U[:, 0].mean()) < 0.05 * vth and np.all(np.abs(U[:, 0]) < 0.15 * vth)


def test_poiseuille_profile_develops():
    """Force-driven flow between diffuse plates (Sec. 5.B): a symmetric,
    near-parabolic velocity profile whose wall friction balances the body
    force in the time average."""
    w = I.channel_poiseuille(ny=32, ppc=100, steps=0)
    sp, ch, dt, st = _setup(w)
    O.channel_step(sp, 0, 7, 0, 2000, ch, dt, st)
    acc = np.zeros(ch.ny * O.NACC + 2)
    nav = 5000
    O.channel_step(sp, 0, 7, 2000, nav, ch, dt, st, acc)
    a = acc[: ch.ny * O.NACC].reshape(ch.ny, O.NACC)
    u = a[:, 1] / a[:, 0]
    yc = (np.arange(ch.ny) + 0.5) * ch.L / ch.ny
    coef = np.polyfit(yc, u, 2)
    fit = np.polyval(coef, yc)
    r2 = 1 - ((u - fit) ** 2).sum() / ((u - u.mean()) ** 2).sum()
    assert r2 > 0.97   # 100 particles per cell: statistical scatter remains
    assert coef[0] < 0                                   # concave
    assert abs(-coef[1] / (2 * coef[0]) / ch.L - 0.5) < 0.05  # vertex at mid-gap
    assert abs(u[: ch.ny // 2].mean() / u[ch.ny // 2:][::-1].mean() - 1) < 0.05
    n = len(st.y)
    wall = acc[ch.ny * O.NACC + 1] / nav
    assert wall == pytest.approx(n * ch.g * dt, rel=0.03)


@pytest.mark.parametrize("form", [0, 1])
def test_channel_fpm_step_is_the_homogeneous_fpm_step_in_one_cell(form):
    """One channel cell, no body force, particles far from the plates (no
    wall event in the step): the channel step with the plain FPM method is the
    homogeneous FPM step at the cell's density n = N F_num / (area L),
    particle for particle, bitwise."""
    w = I.channel_poiseuille()
    rng = np.random.default_rng(17)
    N = 2500
    p = I.equilibrium_particles(rng, N, w.species["m"], w.species["theta_v"], U=(30.0, 0.0, -8.0),
                                T_tr=2500.0, T_rot=600.0, T_vib=1200.0)
    L = 1.0
    F_num = 1e23 * L / N
    ch = O.channel(ny=1, L=L, T_wall=300.0, g=0.0, F_num=F_num, area=1.0, reconstruct=1, method=1)
    sp = O.species(**w.species)
    dt = 0.6 * O.tau_c(sp, 1e23, 2500.0)
    y = rng.uniform(0.45, 0.55, N)
    st = O.ChannelState.from_arrays(y, p.cx, p.cy, p.cz, p.erot, p.lev)
    _, fl, cnt = O.channel_step(sp, form, 5, 2, 1, ch, dt, st)
    assert cnt[O.C_WALL_HITS] == 0
    hs = O.State.from_arrays(p.cx, p.cy, p.cz, p.erot, p.lev)
    O.homog_step_fpm(sp, form, 5, 2, 1, np.array([0, N]), np.array([1e23]), np.array([dt]), hs)
    for a, b in ((st.cx, hs.cx), (st.cy, hs.cy), (st.cz, hs.cz), (st.erot, hs.erot)):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(st.lev, hs.lev)
