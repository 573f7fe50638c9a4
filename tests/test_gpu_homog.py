"""GPU parity of the homogeneous USP-FPM step (CUDA library via the C ABI)
against the FP64 CPU oracle on the same seeded inputs.

Bars (from the method's stated accuracy targets): cell moments within 1e-5
relative (temperatures, Pi) or 1e-5 of the thermal scale (velocities, heat
fluxes); vibrational levels mismatching in fewer than 1e-5 of the particles;
per-cell momentum and total energy conserved to 1e-12 relative in the FP64
form.  In the FP64 form both sides take every discrete decision in double, so
the states must agree to rounding; in the FP32 form the single-step state is
compared within FP32 rounding of the particle arithmetic.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I
from paper_2508_05642_gb300 import usp

pytestmark = pytest.mark.gpu


def _oracle_dt(w):
    sp = O.species(**w.species)
    return np.array([w.dt_over_tau_c * O.tau_c(sp, w.ndens[i], w.T_nominal[i, 0])
                     for i in range(w.n_cells)])


def _gpu_dt(w):
    return np.array([w.dt_over_tau_c * usp.usp_tau_c(w.species, w.ndens[i], w.T_nominal[i, 0])
                     for i in range(w.n_cells)])


def _run_pair(w, steps, precision, tile=0, use_graph=True, particles=None):
    p = particles if particles is not None else w.particles
    form = 1 if precision == usp.USP_FP32 else 0
    if form == 1:
        p = p.astype_f32_exact()
    st = O.State.from_arrays(p.cx, p.cy, p.cz, p.erot, p.lev)
    sp = O.species(**w.species)
    ofl, ocnt = O.homog_step(sp, form, w.seed, 0, steps, w.offsets, w.ndens, _oracle_dt(w), st)
    ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, _gpu_dt(w), p.cx, p.cy, p.cz,
                                   p.erot, p.lev, precision=precision, seed=w.seed, tile=tile,
                                   use_graph=use_graph)
    usp.usp_step(ctx, steps)
    gm = usp.usp_moments(ctx)
    gs = usp.usp_get_particles(ctx)
    gfl, gcnt = usp.usp_status(ctx)
    om = O.moments(sp, w.offsets, st)
    return dict(ctx=ctx, gm=gm, gs=gs, gfl=gfl, gcnt=gcnt, om=om, ost=st, ofl=ofl, ocnt=ocnt, sp=sp)


def _check_moments(om, gm, sp, rel=1e-5, mask=None):
    R = O.R(sp)
    ok = om[0] >= 2 if mask is None else mask
    assert np.array_equal(om[0], gm[0])
    T = om[4][ok]
    vth = np.sqrt(R * T)
    for f in (4, 5):
        np.testing.assert_allclose(gm[f][ok], om[f][ok], rtol=rel, atol=0)
    # T_vib: absolute tolerance scaled by theta_v (T_vib -> 0 at low excitation)
    np.testing.assert_allclose(gm[6][ok], om[6][ok], rtol=rel, atol=rel * 10)
    for f in (1, 2, 3):
        assert np.all(np.abs(gm[f][ok] - om[f][ok]) <= rel * vth)
    for f in range(7, 13):
        assert np.all(np.abs(gm[f][ok] - om[f][ok]) <= rel * R * T)
    for f in range(13, 22):
        scale = vth ** 3 if f < 19 else vth * R * sp.theta_v * max(1.0, 1.0)
        assert np.all(np.abs(gm[f][ok] - om[f][ok]) <= rel * scale * 10)


def test_fp64_single_cell_full_run_matches_oracle():
    """Config-1 workload (1 cell, 20,000 particles, 200 steps, FP64 plain)."""
    w = I.homogeneous_single(N=20000, steps=200)
    r = _run_pair(w, 200, usp.USP_FP64)
    _check_moments(r["om"], r["gm"], r["sp"])
    gx, gy, gz, ge, gl = r["gs"]
    st = r["ost"]
    R = O.R(r["sp"])
    vth = math.sqrt(R * r["om"][4, 0])
    assert np.mean(gl != st.lev) < 1e-5
    if np.all(gl == st.lev):
        assert np.max(np.abs(gx - st.cx)) < 1e-8 * vth
        assert np.max(np.abs(ge - st.erot)) < 1e-8 * R * r["om"][5, 0]
    assert r["gfl"] == r["ofl"]
    assert r["gcnt"][usp.C_CHOL_FIX] == r["ocnt"][O.C_CHOL_FIX] // 20000


def test_fp64_batched_multi_tile_ragged_matches_oracle():
    """Many cells of uneven size; small tiles so cells span several tiles
    with ragged tails; includes cells of 0, 1, 2 and 3 particles."""
    w = I.batched_instances(seed=7, n_inst=40, nmin=50, nmax=3000, steps=10)
    counts = np.diff(w.offsets)
    counts[:4] = [0, 1, 2, 3]
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    rng = np.random.default_rng(8)
    sp = w.species
    parts = [I.equilibrium_particles(rng, int(n), sp["m"], sp["theta_v"], T_tr=w.T_nominal[i, 0],
                                     T_rot=w.T_nominal[i, 1], T_vib=w.T_nominal[i, 2])
             for i, n in enumerate(counts)]
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])
    w.offsets = off
    w.particles = I.Particles(cat("cx"), cat("cy"), cat("cz"), cat("erot"), cat("lev"))
    r = _run_pair(w, 10, usp.USP_FP64, tile=256)
    _check_moments(r["om"], r["gm"], r["sp"])
    gl = r["gs"][4]
    assert np.mean(gl != r["ost"].lev) < 1e-5
    # cells with fewer than two particles are untouched
    for i in range(2):
        b, e = off[i], off[i + 1]
        assert np.array_equal(r["gs"][0][b:e], w.particles.cx[b:e])


def test_fp32_single_step_matches_oracle():
    """FP32 state form, one step from the identical state (the oracle takes
    the level decisions in float, as the kernel does)."""
    w = I.batched_instances(seed=9, n_inst=24, nmin=500, nmax=20000, steps=1)
    r = _run_pair(w, 1, usp.USP_FP32, tile=1024)
    _check_moments(r["om"], r["gm"], r["sp"])
    gx, gy, gz, ge, gl = r["gs"]
    st = r["ost"]
    assert np.mean(gl != st.lev) < 1e-5
    R = O.R(r["sp"])
    for i in range(w.n_cells):
        b, e = w.offsets[i], w.offsets[i + 1]
        vth = math.sqrt(R * r["om"][4, i])
        assert np.max(np.abs(gx[b:e] - st.cx[b:e])) < 2e-5 * vth
        assert np.max(np.abs(gz[b:e] - st.cz[b:e])) < 2e-5 * vth
        eth = R * r["om"][5, i]
        assert np.max(np.abs(ge[b:e] - st.erot[b:e])) < 2e-5 * eth * 20


def test_fp32_multi_step_field_error_is_small():
    """Over 20 steps the FP32 form's cell temperatures stay within 1e-4 of
    the FP64 oracle (the stated FP32-form field error; trajectories
    de-correlate only through rare level flips)."""
    w = I.batched_instances(seed=10, n_inst=16, nmin=2000, nmax=20000, steps=20)
    r = _run_pair(w, 20, usp.USP_FP32)
    om, gm = r["om"], r["gm"]
    for f in (4, 5):
        assert np.max(np.abs(gm[f] / om[f] - 1)) < 1e-4
    assert np.max(np.abs(gm[6] - om[6]) / np.maximum(om[6], 100.0)) < 1e-3


@pytest.mark.parametrize("precision,steps", [(usp.USP_FP64, 4), (usp.USP_FP32, 1)])
def test_every_particle_pass_variant_matches_oracle(precision, steps):
    """The block-tiled and the warp-tiled particle pass at each register
    budget, forced in turn, against one oracle run: cells of 2 to 6000
    particles, so that cells span several tiles of either size with ragged
    tails."""
    w = I.batched_instances(seed=21, n_inst=30, nmin=2, nmax=6000, steps=steps)
    form = 1 if precision == usp.USP_FP32 else 0
    p = w.particles.astype_f32_exact() if form else w.particles
    st = O.State.from_arrays(p.cx, p.cy, p.cz, p.erot, p.lev)
    sp = O.species(**w.species)
    O.homog_step(sp, form, w.seed, 0, steps, w.offsets, w.ndens, _oracle_dt(w), st)
    om = O.moments(sp, w.offsets, st)
    for wt in (0, 1):
        for mb in (2, 3, 4):
            ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, _gpu_dt(w), p.cx, p.cy,
                                           p.cz, p.erot, p.lev, precision=precision,
                                           seed=w.seed, use_graph=True)
            usp.usp_set_variant(ctx, wt, mb)
            assert usp.usp_tuning(ctx)[0] == (wt, mb)
            usp.usp_step(ctx, steps)
            gm = usp.usp_moments(ctx)
            gl = usp.usp_get_particles(ctx)[4]
            flags, _ = usp.usp_status(ctx)
            ctx.destroy()
            assert flags & usp.ERROR_FLAGS == 0, (wt, mb)
            _check_moments(om, gm, sp)
            assert np.mean(gl != st.lev) < 1e-5, (wt, mb)


def test_conservation_on_gpu_fp64():
    w = I.batched_instances(seed=11, n_inst=8, nmin=1000, nmax=5000, steps=0)
    sp = O.species(**w.species)
    R = O.R(sp)
    p = w.particles
    ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, _gpu_dt(w), p.cx, p.cy, p.cz,
                                   p.erot, p.lev, precision=usp.USP_FP64, seed=3)

    def tot(x, y, z, e, l):
        out = []
        for i in range(w.n_cells):
            b, f = w.offsets[i], w.offsets[i + 1]
            out.append((np.array([x[b:f].sum(), y[b:f].sum(), z[b:f].sum()]),
                        (0.5 * (x[b:f] ** 2 + y[b:f] ** 2 + z[b:f] ** 2) + e[b:f]
                         + R * sp.theta_v * l[b:f]).sum(),
                        np.sqrt((x[b:f] ** 2).sum())))
        return out

    t0 = tot(p.cx, p.cy, p.cz, p.erot, p.lev)
    usp.usp_step(ctx, 25)
    t1 = tot(*usp.usp_get_particles(ctx))
    for (m0, e0, v0), (m1, e1, _) in zip(t0, t1):
        assert np.max(np.abs(m1 - m0)) <= 1e-11 * v0
        assert e1 == pytest.approx(e0, rel=1e-12)


def test_graph_and_eager_paths_agree_and_are_deterministic():
    w = I.batched_instances(seed=12, n_inst=8, nmin=500, nmax=4000, steps=0)
    p = w.particles
    outs = []
    for g in (True, False, True):
        ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, _gpu_dt(w), p.cx, p.cy,
                                       p.cz, p.erot, p.lev, precision=usp.USP_FP32, seed=5,
                                       use_graph=g)
        usp.usp_step(ctx, 37)
        outs.append(usp.usp_get_particles(ctx))
        assert usp.usp_launch_count(ctx) >= 74
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    for a, b in zip(outs[0], outs[2]):
        assert np.array_equal(a, b)


def test_step_host_matches_device_path():
    w = I.batched_instances(seed=13, n_inst=6, nmin=500, nmax=3000, steps=0)
    p = w.particles.astype_f32_exact()
    dt = _gpu_dt(w)
    ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz, p.erot,
                                   p.lev, precision=usp.USP_FP32, seed=4)
    usp.usp_step(ctx, 5)
    ref = usp.usp_moments(ctx)
    ctx2 = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz, p.erot,
                                    p.lev, precision=usp.USP_FP32, seed=4)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    mom = np.zeros((usp.USP_NMOM, w.n_cells))
    # The host path works on runs of cells as they arrive, so the particles of
    # a cell are split into other per-block and per-warp partial sums than on
    # the device path: FP32 partials, added in FP64.  No step: the moments of
    # the uploaded state agree to FP32 rounding of those partials.
    usp.usp_step_host(ctx2, f32(p.cx), f32(p.cy), f32(p.cz), f32(p.erot), p.lev, 0, mom)
    ctx0 = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, dt, p.cx, p.cy, p.cz, p.erot,
                                    p.lev, precision=usp.USP_FP32, seed=4)
    _check_moments(usp.usp_moments(ctx0), mom, O.species(**w.species), rel=1e-7)
    # five steps: the FP32 particle arithmetic carries those differences of
    # the cell coefficients to the parity bar of the FP32 form
    usp.usp_step_host(ctx2, f32(p.cx), f32(p.cy), f32(p.cz), f32(p.erot), p.lev, 5, mom)
    _check_moments(ref, mom, O.species(**w.species))


def test_pb_clamp_flag_matches_oracle():
    """A time step close to the limit 2 mu/p = Pr dt drives alpha to 0 and
    p_B = (1 + e_rel)(1 - alpha^2) above 1 (Sec. 3.A.2): both sides clamp the
    binomial and report it."""
    w = I.homogeneous_single(N=5000, T_tr=6000.0, T_rot=6000.0, T_vib=6000.0, steps=1)
    sp = O.species(**w.species)
    T = 6000.0
    mu_p = O.mu(sp, T) / (1e23 * 1.380649e-23 * T)
    w.dt_over_tau_c = 0.97 * 2 * mu_p / O.prandtl(sp, T) / O.tau_c(sp, 1e23, T)
    r = _run_pair(w, 1, usp.USP_FP64)
    assert r["ofl"] & O.F_PB_CLAMP
    assert r["gfl"] & usp.F_PB_CLAMP
    assert r["gcnt"][usp.C_PB_CLAMP] == r["ocnt"][O.C_PB_CLAMP]
    assert np.mean(r["gs"][4] != r["ost"].lev) < 1e-5


@pytest.mark.parametrize("f, lo, hi", [(0.3, 0.5, 1.0), (0.97, 1.0, 10.0)])
def test_fp32_flipped_and_clamped_binomial_match_oracle(f, lo, hi):
    """FP32 table path at p_B above 1/2 (the binomial row taken at 1 - p_B,
    outcome n - k, Sec. 3.A.2) and above 1 (clamped to n and counted): the
    levels equal the oracle's float-decision levels and the clamp counts
    agree.  The time step sets 1 - alpha^2 (alpha -> 0 as Pr dt -> 2 mu/p);
    p_B = (1 + ebar)(1 - alpha^2) at the equilibrium ebar of 6000 K."""
    T = 6000.0
    w = I.homogeneous_single(N=30000, T_tr=T, T_rot=T, T_vib=T, steps=1)
    sp = O.species(**w.species)
    n = float(w.ndens[0])
    mu_p = O.mu(sp, T) / (n * 1.380649e-23 * T)
    w.dt_over_tau_c = f * 2 * mu_p / O.prandtl(sp, T) / O.tau_c(sp, n, T)
    cc = O.cell_coeffs(sp, n, w.dt_over_tau_c * O.tau_c(sp, n, T), T, T, T)
    p_b = (1.0 + 1.0 / math.expm1(sp.theta_v / T)) * (1.0 - cc.alpha ** 2)
    assert lo < p_b < hi
    r = _run_pair(w, 1, usp.USP_FP32)
    assert np.mean(r["gs"][4] != r["ost"].lev) < 1e-5
    assert r["gcnt"][usp.C_PB_CLAMP] == r["ocnt"][O.C_PB_CLAMP]
    if hi > 1.0 + 1e-9 and lo >= 1.0:
        assert r["gfl"] & usp.F_PB_CLAMP and r["ocnt"][O.C_PB_CLAMP] > 0
    else:
        assert r["ocnt"][O.C_PB_CLAMP] == 0
    _check_moments(r["om"], r["gm"], r["sp"])


def test_torch_allocator_path():
    torch = pytest.importorskip("torch")
    w = I.batched_instances(seed=14, n_inst=4, nmin=500, nmax=2000, steps=0)
    p = w.particles
    alloc = usp.torch_allocator()
    ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, _gpu_dt(w), p.cx, p.cy, p.cz,
                                   p.erot, p.lev, precision=usp.USP_FP32, seed=2,
                                   allocator=alloc,
                                   stream=torch.cuda.current_stream().cuda_stream)
    usp.usp_step(ctx, 3)
    m = usp.usp_moments(ctx)
    assert np.all(m[4] > 0)
    ctx.destroy()


def test_fp32_hot_levels_match_oracle():
    """Equilibrium at 20,000 K: mean level ~5.5, levels beyond the kernel's
    per-cell jump tables (32 rows x 48 values) occur, so both the table scan
    and its sequential fallback are exercised; every level must equal the
    oracle's float-decision result."""
    w = I.homogeneous_single(N=60000, T_tr=20000.0, T_rot=20000.0, T_vib=20000.0, steps=1)
    r = _run_pair(w, 1, usp.USP_FP32)
    gl = r["gs"][4]
    assert gl.max() > 48
    assert np.mean(gl != r["ost"].lev) < 1e-5
    _check_moments(r["om"], r["gm"], r["sp"])


def test_moments_of_dyadic_states_are_bitwise_equal():
    """FP64 form, cells of 2^k <= 1024 particles with dyadic-rational
    velocities (multiples of 1/8 below 32 in magnitude), energies and small
    levels: N, U and Pi (sums of at most 52-bit terms) are exact in FP64 in any
    order, so the GPU's equal the oracle's bit for bit; the heat fluxes (cubes)
    agree to rounding."""
    sp_d = I.n2_vhs_relaxation_species()
    sp = O.species(**sp_d)
    rng = np.random.default_rng(5)
    sizes = [2, 4, 8, 16, 32, 64, 128, 256, 1024] * 3
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    d = lambda: rng.integers(-256, 256, n) / 8.0
    cx, cy, cz = d(), d(), d()
    er = np.abs(d()) * 1024
    lev = rng.integers(0, 3, n).astype(np.int32)
    ndens = np.full(len(sizes), 1e23)
    dt = np.full(len(sizes), 1e-9)
    ctx = usp.usp_init_homogeneous(sp_d, off, ndens, dt, cx, cy, cz, er, lev,
                                   precision=usp.USP_FP64, seed=1, tile=256)
    gm = usp.usp_moments(ctx)
    om = O.moments(sp, off, O.State.from_arrays(cx, cy, cz, er, lev))
    for f in list(range(0, 4)) + list(range(7, 13)):
        assert np.array_equal(gm[f], om[f]), f
    np.testing.assert_allclose(gm[4], om[4], rtol=1e-15)
    np.testing.assert_allclose(gm[5], om[5], rtol=1e-15)
    np.testing.assert_allclose(gm[6], om[6], rtol=1e-13)
    scale = np.abs(om[13:22]).max(axis=1, keepdims=True)
    assert np.all(np.abs(gm[13:22] - om[13:22]) <= 1e-13 * scale)


def test_full_size_batched_fp32_sampled_instances_match_oracle():
    """The benchmark configuration (4096 instances, 154M particles, FP32 state,
    autotuned register budget, graph-replayed steps): after 5 steps, sampled
    instances (the smallest, the largest and four others) against the oracle
    run on those instances alone, with the same particle ids and cell index."""
    w = I.batched_instances(seed=1, n_inst=4096, steps=5)
    p = w.particles
    ctx = usp.usp_init_homogeneous(w.species, w.offsets, w.ndens, _gpu_dt(w), p.cx, p.cy, p.cz,
                                   p.erot, p.lev, precision=usp.USP_FP32, seed=w.seed,
                                   use_graph=True)
    usp.usp_step(ctx, 5)
    gm = usp.usp_moments(ctx)
    flags, _ = usp.usp_status(ctx)
    assert flags & usp.ERROR_FLAGS == 0
    ctx.destroy()
    sizes = np.diff(w.offsets)
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 1, 1000, 2048, 4095})
    sp = O.species(**w.species)
    dto = _oracle_dt(w)
    p32 = p.astype_f32_exact()
    for k in sample:
        b, e = int(w.offsets[k]), int(w.offsets[k + 1])
        st = O.State.from_arrays(p32.cx[b:e], p32.cy[b:e], p32.cz[b:e], p32.erot[b:e],
                                 p32.lev[b:e], pid=np.arange(b, e, dtype=np.uint32))
        # cells 0..k-1 empty: the cell streams (I_Delta, +-1 picks) are keyed
        # by the cell index, so the instance keeps its index k
        off = np.zeros(k + 2, dtype=np.int64)
        off[k + 1] = e - b
        O.homog_step(sp, 1, w.seed, 0, 5, off, w.ndens[:k + 1], dto[:k + 1], st)
        om = O.moments(sp, off, st)[:, k]
        g = gm[:, k]
        assert g[0] == om[0]
        for f in (4, 5):
            assert g[f] == pytest.approx(om[f], rel=1e-4), (k, f)
        assert abs(g[6] - om[6]) < 1e-3 * max(om[6], 100.0), k
        vth = math.sqrt(O.R(sp) * om[4])
        assert np.all(np.abs(g[1:4] - om[1:4]) < 1e-4 * vth), k
