"""Pathwise gradients of the channel's time-averaged profiles with respect to
(Z_rot, omega, T_wall), behind a torch.autograd.Function.

The library's tangent forms run every kernel of the channel step on numbers
carrying their derivatives with respect to the three parameters, under the
same random numbers as the plain run of the same precision -- FP64 throughout
(USP_FP64_TANGENT), or FP32 particle values and derivatives with FP64 cell
quantities and accumulation (USP_FP32_TANGENT); discrete outcomes, wall-event
times and particle positions are held (usp.h, usp_backward).  The profiles, their
derivatives and the contraction of those with an objective's gradient are
formed on the device (usp_profiles, usp_backward); this module only marshals
tensors and runs the steps, checkpointing the context (usp_save) every
``checkpoint_every`` steps so that a long run can be resumed (usp_load) from
its last checkpoint instead of from the start.
"""
from __future__ import annotations

import numpy as np

from . import usp

# fields of usp_profiles
PROF_N, PROF_UX, PROF_UY, PROF_UZ, PROF_TTR, PROF_TROT, PROF_TVIB = range(usp.USP_NPROF)


class ChannelGradient:
    """A gradient-form run of the channel: ``warmup`` steps, then ``sample``
    steps whose post-step states are pooled into the time averages.
    theta = (Z_rot, omega, T_wall)."""

    def __init__(self, workload, dt: float, warmup: int, sample: int, seed: int = 1,
                 checkpoint_every: int = 100, keep_checkpoints: bool = False,
                 batches: int = 1, precision: int = usp.USP_FP64_TANGENT):
        if precision not in usp.TANGENT_FORMS:
            raise ValueError("precision must be USP_FP64_TANGENT or USP_FP32_TANGENT")
        self.precision = precision
        self.w = workload
        self.dt = float(dt)
        self.warmup, self.sample = int(warmup), int(sample)
        self.seed = seed
        self.every = max(1, int(checkpoint_every))
        self.keep = keep_checkpoints
        self.batches = max(1, int(batches))
        if self.sample % self.batches:
            raise ValueError("sample must be a multiple of batches")
        self.checkpoints = {}     # step -> host buffer (all of them when keep_checkpoints)
        self.batch_blocks = {}    # end step of a batch -> usp_profiles blocks of that batch
        self.ctx = None
        self.theta = None

    def _create(self, theta):
        sp = dict(self.w.species)
        sp["Z_rot"], sp["omega"] = float(theta[0]), float(theta[1])
        ch = dict(self.w.channel)
        ch["T_wall"] = float(theta[2])
        p = self.w.particles
        return usp.usp_init_channel(sp, ch, self.dt, self.w.y, p.cx, p.cy, p.cz, p.erot, p.lev,
                                    precision=self.precision, seed=self.seed)

    def _advance(self, ctx, start: int):
        """Steps start .. warmup + sample, sampling on from step warmup, a
        checkpoint at every multiple of the checkpoint interval.  With
        batches > 1 the sampling window is cut into equal batches: at the end
        of each, its profiles (and derivatives) are kept and the sums restart
        (batch means give the statistical error of a time average)."""
        total = self.warmup + self.sample
        blen = self.sample // self.batches
        s = start
        while s < total:
            if s == self.warmup:
                usp.usp_channel_sample(ctx, True)
            nxt = min(total, (s // self.every + 1) * self.every)
            if s < self.warmup:
                nxt = min(nxt, self.warmup)
            elif self.batches > 1:
                nxt = min(nxt, self.warmup + ((s - self.warmup) // blen + 1) * blen)
            usp.usp_step(ctx, nxt - s)
            s = nxt
            if self.batches > 1 and s > self.warmup and (s - self.warmup) % blen == 0:
                self.batch_blocks[s] = usp.usp_profiles(ctx)
                usp.usp_sample_read(ctx, reset=True)
            if s % self.every == 0 and s < total:
                buf = usp.usp_save(ctx)
                if not self.keep:
                    self.checkpoints.clear()
                self.checkpoints[s] = buf
        flags, _ = usp.usp_status(ctx)
        if flags & usp.ERROR_FLAGS:
            raise RuntimeError(f"channel run reported errors: flags {flags:#x}")

    def run(self, theta):
        """Run from the initial state; returns the profiles (USP_NPROF x ny)."""
        self.release()
        self.theta = np.asarray(theta, dtype=np.float64).reshape(3)
        self.checkpoints = {}
        self.batch_blocks = {}
        self.ctx = self._create(self.theta)
        self._advance(self.ctx, 0)
        return self.profiles()

    def resume(self, theta, step: int, checkpoint=None):
        """Continue from the checkpoint taken after ``step`` steps (a fresh
        context loads it) to the end of the run; returns the profiles."""
        self.release()
        self.theta = np.asarray(theta, dtype=np.float64).reshape(3)
        buf = self.checkpoints[step] if checkpoint is None else checkpoint
        self.batch_blocks = {k: v for k, v in self.batch_blocks.items() if k <= step}
        self.ctx = self._create(self.theta)
        usp.usp_load(self.ctx, buf)
        self._advance(self.ctx, step)
        return self.profiles()

    def profiles(self):
        return usp.usp_profiles(self.ctx)[0]

    def jacobian(self):
        """d profiles / d theta: (USP_NPROF, ny, 3)."""
        blocks = usp.usp_profiles(self.ctx)
        return np.moveaxis(blocks[1:], 0, -1)

    def batch_results(self):
        """Per batch (ascending end step): profiles (USP_NPROF, ny) and their
        Jacobian (USP_NPROF, ny, 3)."""
        return [(self.batch_blocks[k][0], np.moveaxis(self.batch_blocks[k][1:], 0, -1))
                for k in sorted(self.batch_blocks)]

    def backward(self, d_dL: int) -> np.ndarray:
        """Gradient (3,) of an objective whose dL/dprofiles sits in device
        memory at d_dL (USP_NPROF x ny doubles)."""
        return usp.usp_backward(self.ctx, d_dL)

    def release(self):
        if self.ctx is not None:
            self.ctx.destroy()
            self.ctx = None


def channel_profiles_fn():
    """The torch.autograd.Function (imported lazily so torch stays optional)."""
    import torch

    class ChannelProfiles(torch.autograd.Function):
        """profiles(theta) -> (USP_NPROF, ny) time-averaged profiles of the
        force-driven channel (usp_profiles field order), differentiable in
        theta = (Z_rot, omega, T_wall) (FP64 tensor of 3).  ``runner`` is a
        ChannelGradient; its context stays alive for the backward pass."""

        @staticmethod
        def forward(ctx, theta, runner):
            prof = runner.run(theta.detach().cpu().double().numpy())
            ctx.runner = runner
            return torch.from_numpy(prof).to(theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            dev = torch.device("cuda", torch.cuda.current_device())
            dL = grad_out.detach().to(device=dev, dtype=torch.float64).contiguous()
            torch.cuda.synchronize(dev)
            g = ctx.runner.backward(dL.data_ptr())
            return torch.from_numpy(g).to(grad_out.device), None

    return ChannelProfiles
