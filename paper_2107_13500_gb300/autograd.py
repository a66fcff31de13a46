"""torch.autograd wrappers over the C ABI: differentiable PW tendencies, a
differentiable periodic halo fill, and a forward-Euler rollout with
checkpointed recomputation (the adjoint use of the stencil in variational
data assimilation).

Forward passes call pw_advect / pw_fill_periodic_halo; backward passes call
pw_advect_adjoint / pw_fold_periodic_halo. PyTorch only supplies the tape,
memory and streams.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint

from . import pw

# forward mode -> adjoint arithmetic
_ADJ_MODE = {"f64": "f64", "paired": "paired", "f32": "f32"}


def _as_field(t, like):
    """t in like's layout (shape, strides, 16-byte phase); copies if needed."""
    if (t.shape == like.shape and t.stride() == like.stride() and t.dtype == like.dtype
            and t.data_ptr() % 16 == like.data_ptr() % 16):
        return t
    f = pw.field_like(like)
    f.copy_(t)
    return f


class PWAdvect(torch.autograd.Function):
    """(u, v, w) -> (su, sv, sw); backward is the hand-written adjoint kernel."""

    @staticmethod
    def forward(ctx, u, v, w, coeffs, nx, ny, mode):
        su, sv, sw = pw.advect(u, v, w, coeffs, nx, ny, mode=mode)
        ctx.save_for_backward(u, v, w)
        ctx.coeffs, ctx.nx, ctx.ny, ctx.mode = coeffs, nx, ny, mode
        return su, sv, sw

    @staticmethod
    def backward(ctx, gsu, gsv, gsw):
        u, v, w = ctx.saved_tensors
        g = [pw.field_like(u) if t is None else _as_field(t, u) for t in (gsu, gsv, gsw)]
        gu, gv, gw = pw.advect_adjoint(u, v, w, ctx.coeffs, ctx.nx, ctx.ny, *g, mode=_ADJ_MODE[ctx.mode])
        return gu, gv, gw, None, None, None, None


class FillPeriodicHalo(torch.autograd.Function):
    """Copy of f with its x/y halo made periodic; backward folds the halo."""

    @staticmethod
    def forward(ctx, f, nx, ny):
        out = pw.field_like(f)
        out.copy_(f)
        pw.fill_periodic_halo(out, nx, ny)
        ctx.nx, ctx.ny = nx, ny
        return out

    @staticmethod
    def backward(ctx, g):
        out = pw.field_like(g)
        out.copy_(g)
        pw.fold_periodic_halo(out, ctx.nx, ctx.ny)
        return out, None, None


def advect(u, v, w, coeffs, nx, ny, mode="f64"):
    return PWAdvect.apply(u, v, w, coeffs, nx, ny, mode)


def euler_step(u, v, w, coeffs, nx, ny, dt, mode="f64"):
    """x <- x + dt * F(x) on the interior, then a periodic halo refill."""
    su, sv, sw = advect(u, v, w, coeffs, nx, ny, mode)
    return tuple(FillPeriodicHalo.apply(f + dt * s, nx, ny) for f, s in zip((u, v, w), (su, sv, sw)))


def rollout(u, v, w, coeffs, nx, ny, dt, steps, mode="f64", checkpoint_every=0):
    """`steps` forward-Euler steps. With checkpoint_every = m > 0 only every
    m-th state is kept for the backward pass; each m-step segment is
    recomputed when its gradient is needed."""
    def segment(n):
        def run(a, b, c):
            for _ in range(n):
                a, b, c = euler_step(a, b, c, coeffs, nx, ny, dt, mode)
            return a, b, c
        return run

    if checkpoint_every <= 0:
        return segment(steps)(u, v, w)
    done = 0
    while done < steps:
        n = min(checkpoint_every, steps - done)
        u, v, w = checkpoint(segment(n), u, v, w, use_reentrant=False)
        done += n
    return u, v, w
