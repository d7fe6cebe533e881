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

from . import GS_ERR_STATE, GsError, gs_last_error, gs_rollout_backward, gs_rollout_forward, gs_step_low_backward, \
    gs_step_low_backward_taped, gs_step_low_forward, gs_step_low_forward_taped, gs_upsample_backward, \
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
    """One LR step (Algorithm 1): (x, v) -> (x', v').  With a tag >= 0 (the
    context keeps step tapes, gs_set_step_tapes) the forward keeps its
    recorded passes under the tag and the backward reverses the latest
    record with that tag without recording the step again; a recomputation
    of the step (checkpointing) records it again under the same tag, and a
    record no longer kept falls back to the recording backward."""

    @staticmethod
    def forward(ctx, gctx, dt, iters, x, v, tag=-1):
        x, v = _c(x), _c(v)
        ox, ov = torch.empty_like(x), torch.empty_like(v)
        ctx.tape = int(tag)
        if ctx.tape >= 0:
            _ok(gctx, gs_step_low_forward_taped(gctx.ctx, x.data_ptr(), v.data_ptr(), ox.data_ptr(), ov.data_ptr(),
                                                float(dt), int(iters), ctx.tape), "gs_step_low_forward_taped")
        else:
            _ok(gctx, gs_step_low_forward(gctx.ctx, x.data_ptr(), v.data_ptr(), ox.data_ptr(), ov.data_ptr(),
                                          float(dt), int(iters)), "gs_step_low_forward")
        ctx.gctx, ctx.dt, ctx.iters = gctx, float(dt), int(iters)
        ctx.save_for_backward(x, v)
        return ox, ov

    @staticmethod
    def backward(ctx, g_ox, g_ov):
        x, v = ctx.saved_tensors
        g_ox = torch.zeros_like(x) if g_ox is None else _c(g_ox)
        g_ov = torch.zeros_like(v) if g_ov is None else _c(g_ov)
        gx, gv = torch.empty_like(x), torch.empty_like(v)
        rc = GS_ERR_STATE
        if ctx.tape >= 0:
            rc = gs_step_low_backward_taped(ctx.gctx.ctx, ctx.tape, g_ox.data_ptr(), g_ov.data_ptr(), gx.data_ptr(),
                                            gv.data_ptr())
        if rc == GS_ERR_STATE:
            rc = gs_step_low_backward(ctx.gctx.ctx, x.data_ptr(), v.data_ptr(), g_ox.data_ptr(), g_ov.data_ptr(),
                                      gx.data_ptr(), gv.data_ptr(), ctx.dt, ctx.iters)
        _ok(ctx.gctx, rc, "gs_step_low_backward")
        return None, None, None, gx, gv, None


def frame(gctx, lr_x, lr_v, hr_x, hr_v, dt, n_sub, iters, tag=-1):
    """n_sub LR steps of dt / n_sub, then one HR frame of dt; tag >= 0: the
    LR steps keep their records for the backward under tags tag, tag + 1,
    ... (when gradients are recorded and the context keeps step tapes)."""
    taped = tag >= 0 and getattr(gctx, "step_tapes", 0) > 0 and torch.is_grad_enabled()
    for k in range(n_sub):
        lr_x, lr_v = StepLowFn.apply(gctx, dt / n_sub, iters, lr_x, lr_v, tag + k if taped else -1)
    hr_x, hr_v = UpsampleFn.apply(gctx, dt, lr_x, lr_v, hr_x, hr_v)
    return lr_x, lr_v, hr_x, hr_v


class RolloutFn(torch.autograd.Function):
    """The whole checkpointed rollout as one operation of the library
    (gs_rollout_forward / gs_rollout_backward): (LR x, LR v, HR x, HR v) at
    the start -> the same after `frames` frames.  The context keeps one
    rollout's checkpoints: the backward belongs to the latest forward."""

    @staticmethod
    def forward(ctx, gctx, dt, frames, n_sub, iters, every, lr_x, lr_v, hr_x, hr_v):
        ins = [_c(t) for t in (lr_x, lr_v, hr_x, hr_v)]
        outs = [torch.empty_like(t) for t in ins]
        _ok(gctx, gs_rollout_forward(gctx.ctx, *[t.data_ptr() for t in ins], dt, frames, n_sub, iters, every,
                                     *[t.data_ptr() for t in outs]), "gs_rollout_forward")
        gctx.rollout_serial = getattr(gctx, "rollout_serial", 0) + 1
        ctx.gctx, ctx.serial = gctx, gctx.rollout_serial
        ctx.shapes = [t.shape for t in ins]
        return tuple(outs)

    @staticmethod
    def backward(ctx, *g_out):
        if ctx.gctx.rollout_serial != ctx.serial:
            raise RuntimeError("the context ran another rollout since this one; its checkpoints are gone")
        dev = next(t.device for t in g_out if t is not None) if any(t is not None for t in g_out) else "cuda"
        g = [torch.zeros(sh, dtype=torch.float32, device=dev) if t is None else _c(t)
             for t, sh in zip(g_out, ctx.shapes)]
        grads = [torch.empty_like(t) for t in g]
        _ok(ctx.gctx, gs_rollout_backward(ctx.gctx.ctx, *[t.data_ptr() for t in g], *[t.data_ptr() for t in grads]),
            "gs_rollout_backward")
        return (None,) * 6 + tuple(grads)


def rollout(gctx, lr_x, lr_v, hr_x, hr_v, dt, frames, n_sub=1, iters=4, checkpoint_every=5, tapes=True,
            native=True):
    """Run `frames` frames.  With checkpoint_every > 0 only the states at
    every checkpoint_every-th frame are kept for the backward pass; each
    segment is recomputed from its checkpoint when the gradient flows
    through it.  native: the library runs the whole rollout and its
    backward (RolloutFn); otherwise torch drives it frame by frame, and with
    tapes the context keeps the taped LR steps of one segment, so the
    backward of each step reverses the passes its recomputation recorded
    instead of recording the step again."""
    if native and checkpoint_every > 0:
        return RolloutFn.apply(gctx, float(dt), int(frames), int(n_sub), int(iters), int(checkpoint_every), lr_x,
                               lr_v, hr_x, hr_v)
    if tapes:
        want = (checkpoint_every if checkpoint_every > 0 else frames) * n_sub
        if getattr(gctx, "step_tapes", 0) < want:
            gctx.set_step_tapes(want)
    state = (lr_x, lr_v, hr_x, hr_v)
    # tags: this rollout's serial, then the step's index in the rollout (a
    # segment's recomputation gives its steps the same tags)
    global _ROLLOUTS
    _ROLLOUTS += 1
    base = (_ROLLOUTS & 0xffffffff) << 24

    def segment(f0, k, *s):
        for j in range(k):
            s = frame(gctx, *s, dt, n_sub, iters, tag=base + (f0 + j) * n_sub if tapes else -1)
        return s

    f = 0
    while f < frames:
        k = min(checkpoint_every, frames - f) if checkpoint_every > 0 else frames - f
        if checkpoint_every > 0 and torch.is_grad_enabled():
            state = torch.utils.checkpoint.checkpoint(segment, f, k, *state, use_reentrant=False)
        else:
            state = segment(f, k, *state)
        f += k
    return state


_ROLLOUTS = 0
