"""The oracle's frozen-discrete channel runs, the reference the pathwise
gradients are checked against (tests/test_gpu_grad.py).

A decision log records every discrete decision of a run and the particle
positions; replaying it makes a run with perturbed parameters follow the base
run's branch.  The pins: recording changes nothing; replaying at the base
parameters reproduces the run bit for bit; with perturbed parameters the
replayed run keeps the base positions and particle order; central
differences of the frozen map are smooth (steps h and h/2 agree to O(h^2)),
while the free-running differences at the same step are dominated by the
jumps the replay removes."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_05642_gb300 import inputs as I

WARM, SAMPLE = 20, 20


def _setup():
    w = I.channel_poiseuille(ny=16, ppc=100, Z_vib=1e14, steps=0)
    dt = w.dt_over_tau_c * O.tau_c(O.species(**w.species), w.n, w.channel["T_wall"])
    th = np.array([w.species["Z_rot"], w.species["omega"], w.channel["T_wall"]])
    return w, dt, th


def _run(w, dt, theta, log=None, mode=None):
    d = dict(w.species)
    d["Z_rot"], d["omega"] = theta[0], theta[1]
    sp = O.species(**d)
    chd = dict(w.channel)
    chd["T_wall"] = theta[2]
    ch = O.channel(**chd)
    p = w.particles
    st = O.ChannelState.from_arrays(w.y, p.cx, p.cy, p.cz, p.erot, p.lev)
    acc = np.zeros(ch.ny * O.NACC + 2)
    if log is None:
        O.channel_step(sp, 0, 1, 0, WARM, ch, dt, st)
        O.channel_step(sp, 0, 1, WARM, SAMPLE, ch, dt, st, acc)
    else:
        getattr(log, mode)()
        O.channel_step_frozen(sp, 0, 1, 0, WARM, ch, dt, st, log)
        O.channel_step_frozen(sp, 0, 1, WARM, SAMPLE, ch, dt, st, log, acc)
    return O.channel_profiles(acc, ch.ny, sp), st


def test_record_and_same_parameter_replay_are_the_plain_run():
    w, dt, th = _setup()
    log = O.DecisionLog()
    p0, s0 = _run(w, dt, th)
    p1, s1 = _run(w, dt, th, log, "record")
    st = log.stats()
    assert st["bits"] > 0 and st["ints"] > 0
    p2, s2 = _run(w, dt, th, log, "replay")
    assert log.stats()["mismatches"] == 0 and log.stats()["overruns"] == 0
    for a, b in ((p0, p1), (p0, p2)):
        assert np.array_equal(a, b)
    for s in (s1, s2):
        assert np.array_equal(s.cx, s0.cx) and np.array_equal(s.lev, s0.lev)
        assert np.array_equal(s.pid, s0.pid) and np.array_equal(s.y, s0.y)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_frozen_differences_are_smooth_and_remove_the_jumps(k):
    w, dt, th = _setup()
    log = O.DecisionLog()
    base, s0 = _run(w, dt, th, log, "record")
    fd = {}
    for h in (1e-3, 5e-4):
        tp, tm = th.copy(), th.copy()
        tp[k] *= 1 + h
        tm[k] *= 1 - h
        pp, sp_ = _run(w, dt, tp, log, "replay")
        assert log.stats()["overruns"] == 0
        pm, _ = _run(w, dt, tm, log, "replay")
        # the replay holds positions, order and levels of the base run
        assert np.array_equal(sp_.y, s0.y) and np.array_equal(sp_.pid, s0.pid)
        assert np.array_equal(sp_.lev, s0.lev)
        fd[h] = (pp - pm) / (2 * h * th[k])
    rows = [4, 5, 1]   # T_tr, T_rot, u_x
    scale = np.abs(fd[5e-4][rows]).max(axis=1, keepdims=True)
    assert np.all(scale > 0)
    # O(h^2) difference between the steps
    assert np.all(np.abs(fd[1e-3][rows] - fd[5e-4][rows]) <= 1e-4 * scale)
    # the free-running quotient at the same step sees the jumps
    tp, tm = th.copy(), th.copy()
    tp[k] *= 1 + 1e-3
    tm[k] *= 1 - 1e-3
    free = (_run(w, dt, tp)[0] - _run(w, dt, tm)[0]) / (2e-3 * th[k])
    assert np.abs(free[rows] - fd[5e-4][rows]).max() > 3 * scale.max()


def test_profiles_follow_the_moment_definitions():
    """O.channel_profiles against the pooled sample means computed from the
    particles of each sampled step directly (two steps, one cell layout)."""
    w, dt, th = _setup()
    sp = O.species(**w.species)
    ch = O.channel(**w.channel)
    p = w.particles
    st = O.ChannelState.from_arrays(w.y, p.cx, p.cy, p.cz, p.erot, p.lev)
    acc = np.zeros(ch.ny * O.NACC + 2)
    per = []
    for s in range(2):
        off, _, _ = O.channel_step(sp, 0, 1, s, 1, ch, dt, st, acc)
        per.append((off.copy(), st.cx.copy(), st.cy.copy(), st.cz.copy(), st.erot.copy()))
    prof = O.channel_profiles(acc, ch.ny, sp)
    R = O.R(sp)
    for c in range(ch.ny):
        cs = [np.concatenate([q[i][q[0][c]:q[0][c + 1]] for q in per]) for i in (1, 2, 3, 4)]
        N = len(cs[0])
        U = np.array([x.mean() for x in cs[:3]])
        ttr = (sum((x ** 2).mean() for x in cs[:3]) - (U ** 2).sum()) / (3 * R)
        assert prof[0, c] == pytest.approx(N / 2)
        assert prof[1, c] == pytest.approx(U[0], rel=1e-12, abs=1e-9)
        assert prof[4, c] == pytest.approx(ttr, rel=1e-10)
        assert prof[5, c] == pytest.approx(cs[3].mean() / R, rel=1e-12)
