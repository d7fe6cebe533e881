"""Differentiable pattern: torch.autograd.Function wrappers around the
reverse-mode entry points of libgs, and a rollout with checkpointed
recomputation.

All tensors are float4 records (n, 4) in float32 on the context's device, in
original particle order; the w component is passed through (inverse mass for
LR positions, id for HR positions) and receives no gradient.  The library
context is used as workspace: its stored state is overwritten by every call.
The context must enqueue on torch's current stream (``Context(...,
stream="torch")``) so tensors produced by torch are ready when the library
reads them.
"""
from __future__ import annotations

import torch
import torch.utils.checkpoint

from . import GsError, gs_last_error, gs_step_low_backward, gs_step_low_forward, gs_upsample_backward, \
    gs_upsample_forward


def _ok(gctx, rc, what):
    if rc != 0:
        raise GsError(rc, f"{what}: {gs_last_error(gctx.ctx)}")


def _c(t):
    return t.detach().contiguous()


class UpsampleFn(torch.autograd.Function):
    """One HR frame (Sec. 4): (LR x, LR v, HR x, HR v) -> (HR x', HR v')."""

    @staticmethod
    def forward(ctx, gctx, dt, lr_x, lr_v, hr_x, hr_v):
        lr_x, lr_v, hr_x, hr_v = _c(lr_x), _c(lr_v), _c(hr_x), _c(hr_v)
        ox, ov = torch.empty_like(hr_x), torch.empty_like(hr_v)
        _ok(gctx, gs_upsample_forward(gctx.ctx, lr_x.data_ptr(), lr_v.data_ptr(), hr_x.data_ptr(), hr_v.data_ptr(),
                                      ox.data_ptr(), ov.data_ptr(), float(dt)), "gs_upsample_forward")
        ctx.gctx, ctx.dt = gctx, float(dt)
        ctx.save_for_backward(lr_x, lr_v, hr_x, hr_v)
        return ox, ov

    @staticmethod
    def backward(ctx, g_ox, g_ov):
        lr_x, lr_v, hr_x, hr_v = ctx.saved_tensors
        g_ox = torch.zeros_like(hr_x) if g_ox is None else _c(g_ox)
        g_ov = torch.zeros_like(hr_v) if g_ov is None else _c(g_ov)
        gX, gV = torch.empty_like(lr_x), torch.empty_like(lr_v)
        gx, gv = torch.empty_like(hr_x), torch.empty_like(hr_v)
        _ok(ctx.gctx, gs_upsample_backward(ctx.gctx.ctx, lr_x.data_ptr(), lr_v.data_ptr(), hr_x.data_ptr(),
                                           hr_v.data_ptr(), g_ox.data_ptr(), g_ov.data_ptr(), gX.data_ptr(),
                                           gV.data_ptr(), gx.data_ptr(), gv.data_ptr(), ctx.dt),
            "gs_upsample_backward")
        return None, None, gX, gV, gx, gv


class StepLowFn(torch.autograd.Function):
    """One LR step (Algorithm 1): (x, v) -> (x', v')."""

    @staticmethod
    def forward(ctx, gctx, dt, iters, x, v):
        x, v = _c(x), _c(v)
        ox, ov = torch.empty_like(x), torch.empty_like(v)
        _ok(gctx, gs_step_low_forward(gctx.ctx, x.data_ptr(), v.data_ptr(), ox.data_ptr(), ov.data_ptr(), float(dt),
                                      int(iters)), "gs_step_low_forward")
        ctx.gctx, ctx.dt, ctx.iters = gctx, float(dt), int(iters)
        ctx.save_for_backward(x, v)
        return ox, ov

    @staticmethod
    def backward(ctx, g_ox, g_ov):
        x, v = ctx.saved_tensors
        g_ox = torch.zeros_like(x) if g_ox is None else _c(g_ox)
        g_ov = torch.zeros_like(v) if g_ov is None else _c(g_ov)
        gx, gv = torch.empty_like(x), torch.empty_like(v)
        _ok(ctx.gctx, gs_step_low_backward(ctx.gctx.ctx, x.data_ptr(), v.data_ptr(), g_ox.data_ptr(),
                                           g_ov.data_ptr(), gx.data_ptr(), gv.data_ptr(), ctx.dt, ctx.iters),
            "gs_step_low_backward")
        return None, None, None, gx, gv


def frame(gctx, lr_x, lr_v, hr_x, hr_v, dt, n_sub, iters):
    """n_sub LR steps of dt / n_sub, then one HR frame of dt."""
    for _ in range(n_sub):
        lr_x, lr_v = StepLowFn.apply(gctx, dt / n_sub, iters, lr_x, lr_v)
    hr_x, hr_v = UpsampleFn.apply(gctx, dt, lr_x, lr_v, hr_x, hr_v)
    return lr_x, lr_v, hr_x, hr_v


def rollout(gctx, lr_x, lr_v, hr_x, hr_v, dt, frames, n_sub=1, iters=4, checkpoint_every=5):
    """Run `frames` frames.  With checkpoint_every > 0 only the states at
    every checkpoint_every-th frame are kept for the backward pass; each
    segment is recomputed from its checkpoint when the gradient flows
    through it."""
    state = (lr_x, lr_v, hr_x, hr_v)

    def segment(k, *s):
        for _ in range(k):
            s = frame(gctx, *s, dt, n_sub, iters)
        return s

    f = 0
    while f < frames:
        k = min(checkpoint_every, frames - f) if checkpoint_every > 0 else frames - f
        if checkpoint_every > 0 and torch.is_grad_enabled():
            state = torch.utils.checkpoint.checkpoint(segment, k, *state, use_reentrant=False)
        else:
            state = segment(k, *state)
        f += k
    return state
