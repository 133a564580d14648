"""torch.autograd over CD rollouts (2D, FP64).

The forward pass steps a :class:`~paper_1104_3516_gb300.cd.CDSystem` with
``cd_step``, saving a checkpoint every ``checkpoint_every`` steps; the
backward pass reloads each checkpoint from the last to the first, re-steps
that segment (the steps are deterministic, so the recomputed steps are the
forward steps bit for bit and the tape records them) and back-propagates
through it newest first with ``cd_adjoint_step``.  Memory: one checkpoint per
segment plus a tape of ``checkpoint_every`` steps; time: about two forward
rollouts plus the adjoint solves.

The derivative is that of the time-step map at the recorded contact states
(see ``cd_adjoint_step`` in ``include/cd_api.h``).
"""
from __future__ import annotations

import torch

from . import cd


class CDRollout(torch.autograd.Function):
    """(x0, v0, omega0, mu) -> (x_T, v_T, omega_T, F_T) after `steps` CD
    steps, F_T the 6 wall forces of the last step (sum of the normal impulses
    on wall k over dt; a floor pressure is F_T[2] over the floor's length).

    ``system`` must have been created with ``tape_steps >= checkpoint_every``;
    ``mu`` is a 0-dim tensor holding the system's friction coefficient (the
    gradient with respect to it is returned there).  The system is left in
    the state after the rollout."""

    @staticmethod
    def forward(ctx, x0, v0, w0, mu, system, steps, checkpoint_every, alpha, max_sweeps):
        if int(system.params.tape_steps) < checkpoint_every:
            raise ValueError("the system's tape_steps is shorter than checkpoint_every")
        if float(mu) != float(system.params.mu):
            raise ValueError("mu must equal the system's friction coefficient")
        system.pos.copy_(x0.detach().reshape(-1))
        system.vel.copy_(v0.detach().reshape(-1))
        system.omega.copy_(w0.detach().reshape(-1))
        segments = []
        done = 0
        forces = [0.0] * 6
        while done < steps:
            m = min(checkpoint_every, steps - done)
            segments.append((system.save_checkpoint(), m))
            st = system.step(m)
            forces = st["last"]["wall_force"]
            done += m
        ctx.final = system.save_checkpoint()
        ctx.system, ctx.segments = system, segments
        ctx.alpha, ctx.max_sweeps = alpha, max_sweeps
        ctx.shapes = (x0.shape, v0.shape, w0.shape)
        ctx.stats = []
        F = torch.tensor(forces, dtype=torch.float64)
        return (system.pos.clone().reshape(x0.shape), system.vel.clone().reshape(v0.shape),
                system.omega.clone().reshape(w0.shape), F)

    @staticmethod
    def backward(ctx, gx, gv, gw, gF):
        s = ctx.system
        gx = torch.zeros_like(s.pos) if gx is None else gx.reshape(-1).contiguous().clone()
        gv = torch.zeros_like(s.vel) if gv is None else gv.reshape(-1).contiguous().clone()
        gw = torch.zeros_like(s.omega) if gw is None else gw.reshape(-1).contiguous().clone()
        wall = None if gF is None else gF.detach().cpu().numpy().reshape(6)
        gmu = 0.0
        for buf, m in reversed(ctx.segments):
            s.load_checkpoint(buf)
            s.step(m, stats=False)
            for _ in range(m):
                gx, gv, gw, st = s.adjoint_step(gx, gv, gw, ctx.alpha, ctx.max_sweeps, dL_dwall_force=wall)
                wall = None            # the wall forces are those of the last step only
                gmu += st["dL_dmu"]
                ctx.stats.append(st)
        s.load_checkpoint(ctx.final)
        xs, vs, ws = ctx.shapes
        gmu_t = torch.tensor(gmu, dtype=torch.float64)
        return gx.reshape(xs), gv.reshape(vs), gw.reshape(ws), gmu_t, None, None, None, None, None


def rollout(system, x0, v0, w0, mu, steps, checkpoint_every=20, alpha=1e-13, max_sweeps=100000):
    """Differentiable rollout; see :class:`CDRollout`."""
    return CDRollout.apply(x0, v0, w0, mu, system, steps, checkpoint_every, alpha, max_sweeps)


__all__ = ["CDRollout", "rollout", "cd"]
