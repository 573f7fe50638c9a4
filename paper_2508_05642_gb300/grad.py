"""Pathwise gradients of the channel's time-averaged profiles with respect to
(Z_rot, omega, T_wall), behind a torch.autograd.Function.

The derivatives come from the library's USP_FP64_TANGENT form: every kernel of
the channel step runs on FP64 numbers carrying their derivatives with respect
to the three parameters, under the same random numbers and with the same
discrete outcomes as the plain FP64 run (levels, cell membership, wall hits,
branches are held fixed).  With three parameters this forward (tangent)
propagation gives the full Jacobian in one run, so the autograd backward is a
contraction of the stored Jacobian with the incoming gradient.
"""
from __future__ import annotations

import numpy as np

from . import usp

KB = 1.380649e-23
NACC = 12


def profiles_from_sums(acc: np.ndarray, ny: int, m: float, blocks: int = 1):
    """Time-averaged T_tr, T_rot and u_x per cell (3 x ny) from the pooled
    sums of usp_channel_read, and, for the gradient form, their derivatives
    (3 x ny x 3) with respect to (Z_rot, omega, T_wall)."""
    R = KB / m
    blk = ny * NACC + 2
    A = acc[:blk][: ny * NACC].reshape(ny, NACC)
    N = A[:, 0]
    S1 = A[:, 1:4]
    S2 = A[:, 4:7].sum(axis=1)
    Se = A[:, 10]
    U = S1 / N[:, None]
    T_tr = (S2 / N - (U ** 2).sum(axis=1)) / (3 * R)
    T_rot = Se / (N * R)
    prof = np.stack([T_tr, T_rot, U[:, 0]])
    if blocks == 1:
        return prof, None
    J = np.zeros((3, ny, 3))
    for k in range(3):
        D = acc[(k + 1) * blk:(k + 2) * blk][: ny * NACC].reshape(ny, NACC)
        dS1 = D[:, 1:4]
        dS2 = D[:, 4:7].sum(axis=1)
        dSe = D[:, 10]
        dU = dS1 / N[:, None]
        J[0, :, k] = (dS2 / N - 2 * (U * dU).sum(axis=1)) / (3 * R)
        J[1, :, k] = dSe / (N * R)
        J[2, :, k] = dU[:, 0]
    return prof, J


def channel_profiles_and_jacobian(theta, workload, dt: float, warmup: int, sample: int,
                                  seed: int = 1):
    """Run the gradient form of the channel: `warmup` steps, then `sample`
    steps averaged.  theta = (Z_rot, omega, T_wall)."""
    sp = dict(workload.species)
    sp["Z_rot"], sp["omega"] = float(theta[0]), float(theta[1])
    ch = dict(workload.channel)
    ch["T_wall"] = float(theta[2])
    p = workload.particles
    ctx = usp.usp_init_channel(sp, ch, dt, workload.y, p.cx, p.cy, p.cz, p.erot, p.lev,
                               precision=usp.USP_FP64_TANGENT, seed=seed)
    try:
        if warmup:
            usp.usp_step(ctx, warmup)
        usp.usp_channel_sample(ctx, True)
        usp.usp_step(ctx, sample)
        acc = usp.usp_channel_read(ctx, blocks=4)
        flags, _ = usp.usp_status(ctx)
    finally:
        ctx.destroy()
    if flags & usp.ERROR_FLAGS:
        raise RuntimeError(f"channel run reported errors: flags {flags:#x}")
    return profiles_from_sums(acc, ch["ny"], sp["m"], blocks=4)


def channel_profiles_fn():
    """The torch.autograd.Function (imported lazily so torch stays optional)."""
    import torch

    class ChannelProfiles(torch.autograd.Function):
        """profiles(theta) -> (3, ny): time-averaged T_tr, T_rot, u_x per cell
        of the force-driven channel, differentiable in theta = (Z_rot, omega,
        T_wall) (0-dim or 1-dim FP64 tensor of 3)."""

        @staticmethod
        def forward(ctx, theta, workload, dt, warmup, sample, seed):
            th = theta.detach().cpu().double().numpy().reshape(3)
            prof, J = channel_profiles_and_jacobian(th, workload, dt, warmup, sample, seed)
            ctx.save_for_backward(torch.from_numpy(J))
            return torch.from_numpy(prof).to(theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            (J,) = ctx.saved_tensors
            g = torch.einsum("fc,fck->k", grad_out.detach().cpu().double(), J)
            return g.to(grad_out.device), None, None, None, None, None

    return ChannelProfiles
