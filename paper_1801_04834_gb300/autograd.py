"""torch.autograd.Function wrappers of the differentiation form.

`correct_correlate(c, chan, gains, delays, bandpass=None, recompute=True)`
runs the hot path forward (fx_correct with the given gains and a delay held
constant over the block, then fx_correlate) and differentiates it with the
hand-written adjoint kernel (fx_correct_correlate_backward). The adjoint
needs the raw visibilities R of the bandpass-corrected data; with
`recompute=True` they are recomputed from the channelised block in the
backward pass (only a reference to `chan`, which the caller holds anyway, is
kept), with `recompute=False` they are formed in the forward pass and kept
(one extra correction + correlation up front, after which `chan` may be
freed: R is ~1/(S/2N) of its size).

With `delays_end` given, each station's delay moves linearly from `delays`
(block start) to `delays_end` (block end), as fx_correct interpolates it;
the visibility no longer factors through R, and the backward pass calls
fx_correct_correlate_backward_interp, which recomputes the corrected block
from `chan` and returns gradients for both ends (the channelised block is
always kept by reference in this mode).

`apply_gains(c, raw_vis, gains, delays)` is the cheap forward from R (for
calibration loops that re-evaluate V for many gains/delays on fixed data).

gains: float32 [N][2][2] (re, im per station and pol); delays: float64 [N]
seconds; the output vis is float32 [SB][C][B][4][2].
"""
from __future__ import annotations

import torch


class _CorrectCorrelate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gains, delays, c, chan, bandpass, recompute):
        g = gains.detach().contiguous()
        d = delays.detach().contiguous()
        vis = c.correlate(c.correct(chan, d, d, bandpass=bandpass, gains=g))
        ctx.c, ctx.bandpass, ctx.recompute = c, bandpass, recompute
        if recompute:
            ctx.chan = chan
            ctx.save_for_backward(g, d)
        else:
            ctx.chan = None
            ctx.save_for_backward(g, d, c.raw_vis(chan, bandpass))
        return vis

    @staticmethod
    def backward(ctx, grad_vis):
        c = ctx.c
        if ctx.recompute:
            g, d = ctx.saved_tensors
            R = c.raw_vis(ctx.chan, ctx.bandpass)
        else:
            g, d, R = ctx.saved_tensors
        gg, gt = c.backward(R, g, d, grad_vis.contiguous())
        return gg, gt, None, None, None, None


class _ApplyGains(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gains, delays, c, raw_vis):
        g = gains.detach().contiguous()
        d = delays.detach().contiguous()
        ctx.c = c
        ctx.save_for_backward(g, d, raw_vis)
        return c.apply_gains(raw_vis, g, d)

    @staticmethod
    def backward(ctx, grad_vis):
        g, d, R = ctx.saved_tensors
        gg, gt = ctx.c.backward(R, g, d, grad_vis.contiguous())
        return gg, gt, None, None


class _CorrectCorrelateInterp(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gains, delays, delays_end, c, chan, bandpass):
        g = gains.detach().contiguous()
        d0 = delays.detach().contiguous()
        d1 = delays_end.detach().contiguous()
        vis = c.correlate(c.correct(chan, d0, d1, bandpass=bandpass, gains=g))
        ctx.c, ctx.chan, ctx.bandpass = c, chan, bandpass
        ctx.save_for_backward(g, d0, d1)
        return vis

    @staticmethod
    def backward(ctx, grad_vis):
        g, d0, d1 = ctx.saved_tensors
        gg, gb, ge = ctx.c.backward_interp(ctx.chan, g, d0, d1, grad_vis.contiguous(), bandpass=ctx.bandpass)
        return gg, gb, ge, None, None, None


def correct_correlate(c, chan, gains, delays, bandpass=None, recompute=True, delays_end=None):
    if delays_end is not None:
        return _CorrectCorrelateInterp.apply(gains, delays, delays_end, c, chan, bandpass)
    return _CorrectCorrelate.apply(gains, delays, c, chan, bandpass, recompute)


def apply_gains(c, raw_vis, gains, delays):
    return _ApplyGains.apply(gains, delays, c, raw_vis)
