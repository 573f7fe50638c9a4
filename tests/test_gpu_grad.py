"""Pathwise gradients of the channel profiles with respect to (Z_rot, omega,
T_wall): the library's derivative (tangent) form, contracted on the device by
usp_backward, against central finite differences of the FP64 CPU oracle on
the Poiseuille gradient workload (64 cells x 200 particles; Z_vib = 1e14 as
in the paper's Poiseuille case, Sec. 5.B, which freezes the vibrational
exchange at 300 K).

The finite differences are taken on the oracle's frozen-discrete form: its
base run records every discrete decision (levels, cell membership, wall
events and their times, branches, +-1 picks) and the particle positions, and
the runs at theta (1 +- 1e-3) replay them, so the quotient differentiates the
same branch the pathwise gradient does.

The forward dynamics is chaotic: the library's FP64 run and the oracle's,
which differ only in rounding (summation order, math-library last bits),
agree to 1e-10 m/s after 100 steps and 2e-4 m/s after 500 (the difference
grows about tenfold per 100 steps), and part ways in their discrete outcomes
soon after.  So

* over 400 steps (200 warm-up, 200 averaged), where the two runs are one
  realization, the derivatives are compared entry by entry at 1e-3 relative;
* over the full 2,000 steps (1,000 warm-up, 1,000 averaged in 10 batches of
  100, checkpoint every 100 steps), the two are different realizations of
  the same pathwise estimator: the objective's gradient is compared by batch
  means within four combined standard errors, and the run is resumed from its
  checkpoints bit for bit."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_05642_gb300 import grad as G
from paper_2508_05642_gb300 import inputs as I

pytestmark = pytest.mark.gpu

H = 1e-3
EVERY = 100
FIELDS = (G.PROF_TTR, G.PROF_TROT, G.PROF_UX)


def _workload():
    return I.channel_poiseuille(ny=64, ppc=200, Z_vib=1e14, steps=0)


def _dt(w):
    return w.dt_over_tau_c * O.tau_c(O.species(**w.species), w.n, w.channel["T_wall"])


def _theta(w):
    return np.array([w.species["Z_rot"], w.species["omega"], w.channel["T_wall"]])


def _weights(ny, nf):
    """The gradient workload's objective: every cell's time-averaged T_tr,
    T_rot and u_x with fixed random weights (seed 2), scaled to O(1)."""
    rng = np.random.default_rng(2)
    wts = np.zeros((nf, ny))
    scl = {G.PROF_TTR: 1 / 300.0, G.PROF_TROT: 1 / 300.0, G.PROF_UX: 1 / 10.0}
    for f in FIELDS:
        wts[f] = rng.uniform(0.5, 1.5, ny) * scl[f]
    return wts


def _oracle_run(w, theta, dt, log, mode, warm, sample, batches=1):
    """Profiles of a frozen-discrete oracle run, one (7, ny) array per batch."""
    d = dict(w.species)
    d["Z_rot"], d["omega"] = theta[0], theta[1]
    sp = O.species(**d)
    chd = dict(w.channel)
    chd["T_wall"] = theta[2]
    ch = O.channel(**chd)
    p = w.particles
    st = O.ChannelState.from_arrays(w.y, p.cx, p.cy, p.cz, p.erot, p.lev)
    getattr(log, mode)()
    _, fl, _ = O.channel_step_frozen(sp, 0, 1, 0, warm, ch, dt, st, log)
    out = []
    blen = sample // batches
    for b in range(batches):
        acc = np.zeros(ch.ny * O.NACC + 2)
        _, f1, _ = O.channel_step_frozen(sp, 0, 1, warm + b * blen, blen, ch, dt, st, log, acc)
        fl |= f1
        out.append(O.channel_profiles(acc, ch.ny, sp))
    st_ = log.stats()
    assert st_["overruns"] == 0
    return out, fl


def _frozen_fd(w, dt, th, warm, sample, batches=1):
    log = O.DecisionLog()
    base, flags = _oracle_run(w, th, dt, log, "record", warm, sample, batches)
    assert flags & (O.F_TREL_CLAMP | O.F_CHOL_FAIL_AFTER_FIX | O.F_NEG_RADICAND) == 0
    fd = [np.zeros(b.shape + (3,)) for b in base]
    for k in range(3):
        tp, tm = th.copy(), th.copy()
        tp[k] *= 1 + H
        tm[k] *= 1 - H
        pp, _ = _oracle_run(w, tp, dt, log, "replay", warm, sample, batches)
        pm, _ = _oracle_run(w, tm, dt, log, "replay", warm, sample, batches)
        for b in range(len(base)):
            fd[b][..., k] = (pp[b] - pm[b]) / (2 * H * th[k])
    return base, fd


# ---------------------------------------------------------------------------
# one realization: 400 steps
# ---------------------------------------------------------------------------
WARM_A, SAMPLE_A = 200, 200


@pytest.fixture(scope="module")
def short():
    w = _workload()
    dt = _dt(w)
    th = _theta(w)
    base, fd = _frozen_fd(w, dt, th, WARM_A, SAMPLE_A)
    r = G.ChannelGradient(w, dt, WARM_A, SAMPLE_A, checkpoint_every=EVERY)
    prof = r.run(th)
    J = r.jacobian()
    r.release()
    return w, dt, th, base[0], fd[0], prof, J


def test_tangent_values_match_fp64_oracle(short):
    """The derivative form takes the FP64 form's decisions: its profiles equal
    the oracle's over the 400 steps."""
    _, _, _, base, _, prof, _ = short
    for f in FIELDS + (G.PROF_N, G.PROF_TVIB):
        np.testing.assert_allclose(prof[f], base[f], rtol=1e-9, atol=1e-9 * np.abs(base[f]).max())


def test_jacobian_matches_frozen_central_differences(short):
    """d(T_tr, T_rot, u_x profiles)/d(Z_rot, omega, T_wall), every cell,
    within 1e-3 relative of the frozen-discrete central differences (an
    absolute floor of 1e-4 of each field's and parameter's largest entry for
    entries that are nearly zero)."""
    _, _, _, _, fd, _, J = short
    for f in FIELDS:
        for k in range(3):
            scale = np.abs(fd[f, :, k]).max()
            err = np.abs(J[f, :, k] - fd[f, :, k])
            assert np.all(err <= 1e-3 * np.abs(fd[f, :, k]) + 1e-4 * scale), \
                (f, k, float(err.max()), float(scale))


def test_backward_and_autograd_match_objective_differences(short):
    """The objective through the torch.autograd.Function: its gradient is
    usp_backward's device contraction, and within 1e-3 relative of the
    objective's frozen-discrete central differences."""
    torch = pytest.importorskip("torch")
    w, dt, th, base, fd, _, J = short
    wts = _weights(base.shape[1], base.shape[0])
    F = G.channel_profiles_fn()
    r = G.ChannelGradient(w, dt, WARM_A, SAMPLE_A, checkpoint_every=EVERY)
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    prof = F.apply(theta, r)
    loss = (torch.from_numpy(wts) * prof).sum()
    loss.backward()
    g = theta.grad.numpy()
    r.release()
    np.testing.assert_allclose(g, np.einsum("fc,fck->k", wts, J), rtol=1e-12)
    np.testing.assert_allclose(g, np.einsum("fc,fck->k", wts, fd), rtol=1e-3)


# ---------------------------------------------------------------------------
# the full 2,000 steps
# ---------------------------------------------------------------------------
WARM_B, SAMPLE_B, BATCHES = 1000, 1000, 10


@pytest.fixture(scope="module")
def long_run():
    w = _workload()
    dt = _dt(w)
    th = _theta(w)
    base, fd = _frozen_fd(w, dt, th, WARM_B, SAMPLE_B, BATCHES)
    r = G.ChannelGradient(w, dt, WARM_B, SAMPLE_B, checkpoint_every=EVERY,
                          keep_checkpoints=True, batches=BATCHES)
    r.run(th)
    yield w, dt, th, base, fd, r
    r.release()


def test_long_run_gradient_agrees_with_oracle_differences(long_run):
    """Batch means of the objective's gradient over the last 1,000 of 2,000
    steps: library (pathwise, its own realization) and oracle (frozen-discrete
    central differences, its own realization) within four combined standard
    errors; where a gradient is resolved (more than four standard errors
    from zero: omega and T_wall here, the Z_rot gradient of this objective is
    zero within its scatter), both standard errors are below 10 % of it."""
    _, _, _, base, fd, r = long_run
    wts = _weights(base[0].shape[1], base[0].shape[0])
    gpu = np.array([np.einsum("fc,fck->k", wts, J) for _, J in r.batch_results()])
    orc = np.array([np.einsum("fc,fck->k", wts, d) for d in fd])
    assert gpu.shape == orc.shape == (BATCHES, 3)
    mg, mo = gpu.mean(axis=0), orc.mean(axis=0)
    sg = gpu.std(axis=0, ddof=1) / np.sqrt(BATCHES)
    so = orc.std(axis=0, ddof=1) / np.sqrt(BATCHES)
    assert np.all(np.abs(mg - mo) <= 4 * np.sqrt(sg ** 2 + so ** 2)), (mg, mo, sg, so)
    resolved = np.abs(mo) > 4 * so
    assert resolved[1] and resolved[2], (mo, so)
    assert np.all((sg < 0.1 * np.abs(mg)) | ~resolved) and np.all((so < 0.1 * np.abs(mo)) | ~resolved)


def test_checkpoint_resume_reproduces_the_run(long_run):
    """Step checkpointing: a fresh context resumed from the checkpoints after
    500 and after 1,500 steps yields the same batches, profiles and
    derivatives bit for bit, as the uninterrupted 2,000-step run."""
    w, dt, th, _, _, r = long_run
    assert sorted(r.checkpoints) == list(range(EVERY, WARM_B + SAMPLE_B, EVERY))
    ref = r.batch_results()
    for step in (500, 1500):
        q = G.ChannelGradient(w, dt, WARM_B, SAMPLE_B, checkpoint_every=EVERY, batches=BATCHES)
        q.batch_blocks = {k: v for k, v in r.batch_blocks.items() if k <= step}
        q.resume(th, step, r.checkpoints[step])
        got = q.batch_results()
        assert len(got) == len(ref)
        for (pa, ja), (pb, jb) in zip(ref, got):
            assert np.array_equal(pa, pb) and np.array_equal(ja, jb)
        q.release()


# ---------------------------------------------------------------------------
# the FP32 gradient form (FP32 particle values and derivatives, FP64 cell
# quantities and accumulation)
# ---------------------------------------------------------------------------
def test_fp32_tangent_values_follow_the_fp32_form():
    """Over the first steps the FP32 gradient form's values are the FP32
    form's (the same float operations carry the values; the derivative slots
    ride along): profiles after 5 + 5 steps within 1e-5 relative."""
    from paper_2508_05642_gb300 import usp
    w = _workload()
    dt = _dt(w)
    r = G.ChannelGradient(w, dt, 5, 5, precision=usp.USP_FP32_TANGENT)
    prof = r.run(_theta(w))
    r.release()
    p = w.particles
    ctx = usp.usp_init_channel(w.species, w.channel, dt, w.y, p.cx, p.cy, p.cz, p.erot, p.lev,
                               precision=usp.USP_FP32, seed=1)
    usp.usp_step(ctx, 5)
    usp.usp_channel_sample(ctx, True)
    usp.usp_step(ctx, 5)
    ref = usp.usp_profiles(ctx)
    ctx.destroy()
    for f in FIELDS:
        np.testing.assert_allclose(prof[f], ref[f], rtol=1e-5, atol=1e-5 * np.abs(ref[f]).max())


def test_fp32_tangent_long_run_gradient_agrees_with_oracle_differences(long_run):
    """The FP32 gradient form over the 2,000 steps (its own realization: FP32
    and FP64 runs of the channel part ways within about 100 steps, and the
    Z_rot and omega derivatives of single cells are dominated by sampling
    noise at this size, so entries are not compared one by one): batch means
    of the objective's gradient within four combined standard errors of the
    oracle's frozen-discrete central differences, omega and T_wall resolved
    to 10 %."""
    from paper_2508_05642_gb300 import usp
    w, dt, th, base, fd, _ = long_run
    r = G.ChannelGradient(w, dt, WARM_B, SAMPLE_B, checkpoint_every=EVERY, batches=BATCHES,
                          precision=usp.USP_FP32_TANGENT)
    r.run(th)
    res = r.batch_results()
    r.release()
    wts = _weights(base[0].shape[1], base[0].shape[0])
    g32 = np.array([np.einsum("fc,fck->k", wts, J) for _, J in res])
    orc = np.array([np.einsum("fc,fck->k", wts, d) for d in fd])
    m32, mo = g32.mean(axis=0), orc.mean(axis=0)
    s32 = g32.std(axis=0, ddof=1) / np.sqrt(BATCHES)
    so = orc.std(axis=0, ddof=1) / np.sqrt(BATCHES)
    assert np.all(np.abs(m32 - mo) <= 4 * np.sqrt(s32 ** 2 + so ** 2)), (m32, mo, s32, so)
    assert np.all(s32[1:] < 0.1 * np.abs(m32[1:])), (m32, s32)
