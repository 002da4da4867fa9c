"""torch.autograd wrappers of the DG residual and of K LSERK steps.

Forward and backward both run in libdg.so: DGRHS.forward is dg_rhs and its
backward dg_rhs_vjp (the hand-written adjoint of Eq. 1's residual); DGRK
advances K LSERK(5,4) steps with dg_rk_step_checkpointed (keeping the state
at the start of every segment of ckpt_every steps) and its backward is
dg_rk_vjp_checkpointed (reverse LSERK recomputing each segment from its
checkpoint).  Tensors are float64 CUDA
tensors in the library's storage layout.
"""
from __future__ import annotations

import torch


class DGRHS(torch.autograd.Function):
    """R = rhs(Q) for a fixed mesh."""

    @staticmethod
    def forward(ctx, Q, mesh):
        Q = Q.contiguous()
        ctx.mesh = mesh
        ctx.save_for_backward(Q)
        return mesh.rhs(Q)

    @staticmethod
    def backward(ctx, Rbar):
        (Q,) = ctx.saved_tensors
        return ctx.mesh.rhs_vjp(Q, Rbar.contiguous()), None


class DGRK(torch.autograd.Function):
    """Q_K after nsteps LSERK steps of size dt from Q0."""

    @staticmethod
    def forward(ctx, Q0, mesh, dt, nsteps, ckpt_every=5):
        Q0 = Q0.contiguous()
        ctx.mesh, ctx.dt, ctx.nsteps, ctx.ckpt = mesh, float(dt), int(nsteps), int(ckpt_every)
        Q = Q0.clone()
        ckpts = mesh.rk_step_checkpointed(Q, torch.empty_like(Q), dt, nsteps, ckpt_every)
        ctx.save_for_backward(ckpts)
        return Q

    @staticmethod
    def backward(ctx, QKbar):
        (ckpts,) = ctx.saved_tensors
        Q0bar = ctx.mesh.rk_vjp_checkpointed(ckpts, ctx.dt, ctx.nsteps, ctx.ckpt, QKbar.contiguous())
        return Q0bar, None, None, None, None


def rhs(Q, mesh):
    return DGRHS.apply(Q, mesh)


def rk(Q0, mesh, dt, nsteps, ckpt_every=5):
    return DGRK.apply(Q0, mesh, dt, nsteps, ckpt_every)
