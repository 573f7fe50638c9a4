"""Pathwise gradients of the channel profiles with respect to (Z_rot, omega,
T_wall): the library's derivative (tangent) form against central finite
differences of the FP64 CPU oracle under the same random numbers.

The finite-difference step is 1e-7 relative, small enough that no discrete
outcome (vibrational level, cell membership, wall hit) changes between the
perturbed oracle runs and the base run -- the test checks that -- so the
difference quotient is the derivative of the same branch the pathwise
gradient differentiates.  Z_vib = 1e14 as in the paper's Poiseuille case
(Sec. 5.B), which freezes the vibrational exchange at 300 K."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_05642_gb300 import grad as G
from paper_2508_05642_gb300 import inputs as I
from paper_2508_05642_gb300 import usp

pytestmark = pytest.mark.gpu

WARM, SAMPLE = 20, 20


def _workload():
    return I.channel_poiseuille(ny=16, ppc=100, Z_vib=1e14, steps=0)


def _dt(w):
    return w.dt_over_tau_c * O.tau_c(O.species(**w.species), w.n, w.channel["T_wall"])


def _oracle_profiles(w, theta, dt, seed=1):
    d = dict(w.species)
    d["Z_rot"], d["omega"] = theta[0], theta[1]
    sp = O.species(**d)
    chd = dict(w.channel)
    chd["T_wall"] = theta[2]
    ch = O.channel(**chd)
    p = w.particles
    st = O.ChannelState.from_arrays(w.y, p.cx, p.cy, p.cz, p.erot, p.lev)
    O.channel_step(sp, 0, seed, 0, WARM, ch, dt, st)
    acc = np.zeros(ch.ny * O.NACC + 2)
    O.channel_step(sp, 0, seed, WARM, SAMPLE, ch, dt, st, acc)
    prof, _ = G.profiles_from_sums(acc, ch.ny, d["m"])
    return prof, st


def test_tangent_values_match_fp64_form():
    w = _workload()
    dt = _dt(w)
    theta = (w.species["Z_rot"], w.species["omega"], w.channel["T_wall"])
    prof_t, J = G.channel_profiles_and_jacobian(theta, w, dt, WARM, SAMPLE)
    prof_o, _ = _oracle_profiles(w, theta, dt)
    np.testing.assert_allclose(prof_t, prof_o, rtol=1e-9, atol=1e-9)
    assert np.all(np.isfinite(J)) and np.abs(J).max() > 0


def test_jacobian_matches_oracle_central_differences():
    w = _workload()
    dt = _dt(w)
    theta = np.array([w.species["Z_rot"], w.species["omega"], w.channel["T_wall"]])
    _, J = G.channel_profiles_and_jacobian(theta, w, dt, WARM, SAMPLE)
    _, st0 = _oracle_profiles(w, theta, dt)
    h = 1e-7
    for k in range(3):
        tp, tm = theta.copy(), theta.copy()
        tp[k] *= 1 + h
        tm[k] *= 1 - h
        pp, sp_ = _oracle_profiles(w, tp, dt)
        pm, sm_ = _oracle_profiles(w, tm, dt)
        # same discrete branch in all three runs
        for s in (sp_, sm_):
            assert np.array_equal(s.pid, st0.pid) and np.array_equal(s.lev, st0.lev)
        fd = (pp - pm) / (2 * h * theta[k])
        scale = np.abs(fd).max(axis=1, keepdims=True)
        err = np.abs(J[:, :, k] - fd)
        assert np.all(err <= 1e-3 * np.abs(fd) + 1e-5 * scale), (k, err.max(), scale.ravel())


def test_autograd_function_backward_is_jacobian_contraction():
    torch = pytest.importorskip("torch")
    w = _workload()
    dt = _dt(w)
    F = G.channel_profiles_fn()
    theta = torch.tensor([w.species["Z_rot"], w.species["omega"], w.channel["T_wall"]],
                         dtype=torch.float64, requires_grad=True)
    prof = F.apply(theta, w, dt, WARM, SAMPLE, 1)
    wts = torch.from_numpy(np.random.default_rng(2).uniform(0.5, 1.5, prof.shape))
    scl = torch.tensor([[1.0 / 300.0], [1.0 / 300.0], [1.0 / 10.0]], dtype=torch.float64)
    loss = (wts * scl * prof).sum()
    loss.backward()
    th = theta.detach().numpy()
    _, J = G.channel_profiles_and_jacobian(th, w, dt, WARM, SAMPLE)
    expect = np.einsum("fc,fck->k", (wts * scl).numpy(), J)
    np.testing.assert_allclose(theta.grad.numpy(), expect, rtol=1e-12)
    # and the objective's gradient against the oracle's central differences
    h = 1e-7
    for k in range(3):
        tp, tm = th.copy(), th.copy()
        tp[k] *= 1 + h
        tm[k] *= 1 - h
        lp = float((wts * scl).numpy().ravel() @ _oracle_profiles(w, tp, dt)[0].ravel())
        lm = float((wts * scl).numpy().ravel() @ _oracle_profiles(w, tm, dt)[0].ravel())
        fd = (lp - lm) / (2 * h * th[k])
        assert theta.grad[k].item() == pytest.approx(fd, rel=1e-3, abs=1e-9 * abs(loss.item()))
