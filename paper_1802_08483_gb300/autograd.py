"""torch.autograd.Function wrappers around the decoder's adjoint path.

forward() runs the decoder on the priors where they live (CUDA priors stay on
the device; the call is issued on torch's current stream).  When an input
needs a gradient it calls mapdec_loglik_grad / mapdec_batch_loglik_grad, whose
CUDA kernels compute log P(Y) together with d logP / d(Pi, Pd, Ps) and
d logP / d prior, and saves the gradients; otherwise it runs the decode path
alone for log P(Y).  backward() scales the saved gradients by the incoming
gradient.  PyTorch only moves the tensors; every step of the computation runs
in libmapdec.so.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import mapdec


def _chan_tuple(chan):
    c = chan.detach().to("cpu", torch.float64).reshape(-1)
    return float(c[0]), float(c[1]), float(c[2])


def _same_channel(got, want) -> bool:
    """chan holds the channel the decoder was planned for (to float32 rounding)."""
    return all(math.isclose(a, b, rel_tol=1e-6, abs_tol=1e-12) for a, b in zip(got, want))


def _on_current_stream(handle, device):
    """Issue the handle's work on torch's current stream of a CUDA device, so
    that it is ordered after the kernels that produced its inputs."""
    if device.type == "cuda":
        handle.set_stream(torch.cuda.current_stream(device).cuda_stream)


class FrameLogLik(torch.autograd.Function):
    """log P(Y) of one frame as a function of (priors (N, q), chan = [Pi, Pd, Ps]).

    The decoder handle carries the code and channel; chan must hold the same
    channel values the handle was created with (the derivative is taken there).
    """

    @staticmethod
    def forward(ctx, priors, chan, decoder, rx):
        if not _same_channel(_chan_tuple(chan), (decoder.Pi, decoder.Pd, decoder.Ps)):
            raise ValueError("chan differs from the decoder's channel parameters")
        dev = priors.device
        pr = priors.detach().to(torch.float32).contiguous()
        ll = torch.zeros(1, dtype=torch.float64, device=dev)
        _on_current_stream(decoder, dev)
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            dpri = torch.empty_like(pr)
            dchan = torch.zeros(3, dtype=torch.float64, device=dev)
            decoder.loglik_grad_into(rx, pr, dchan, dpri, ll)
            ctx.save_for_backward(dpri, dchan.to(chan.device))
        else:
            decoder.loglik_into(rx, pr, ll)
        ctx.dtypes = (priors.dtype, chan.dtype)
        return ll[0]

    @staticmethod
    def backward(ctx, grad_out):
        dpri, dchan = ctx.saved_tensors
        g = grad_out.to(torch.float64)
        gp = (dpri.to(torch.float64) * g).to(ctx.dtypes[0]) if ctx.needs_input_grad[0] else None
        gc = (dchan * g.to(dchan.device)).to(ctx.dtypes[1]) if ctx.needs_input_grad[1] else None
        return gp, gc, None, None


class BatchLogLik(torch.autograd.Function):
    """Per-frame log P(Y) of a batch (created with MAPDEC_BATCH_GRAD) as a
    function of the concatenated priors (flat, as in mapdec_batch_layout) and
    the per-frame channel parameters chan (num_frames, 3)."""

    @staticmethod
    def forward(ctx, priors_all, chan, batch, rx_all):
        ch = chan.detach().to("cpu", torch.float64).reshape(-1)
        if ch.numel() != 3 * len(batch.frames):
            raise ValueError(f"chan holds {ch.numel()} values for {len(batch.frames)} frames")
        for k, f in enumerate(batch.frames):
            got = (float(ch[3 * k]), float(ch[3 * k + 1]), float(ch[3 * k + 2]))
            if not _same_channel(got, (f.Pi, f.Pd, f.Ps)):
                raise ValueError(f"chan of frame {k} differs from the batch's channel parameters")
        dev = priors_all.device
        pr = priors_all.detach().to(torch.float32).contiguous()
        nf = len(batch.frames)
        ll = torch.zeros(nf, dtype=torch.float64, device=dev)
        rx = np.ascontiguousarray(rx_all, np.uint8)
        _on_current_stream(batch, dev)
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            dpri = torch.empty_like(pr)
            dchan = torch.zeros(nf, 3, dtype=torch.float64, device=dev)
            st = batch.loglik_grad_into(rx, pr, dchan, dpri, ll)
            if st != 0:
                raise mapdec.MapDecError(st, "mapdec_batch_loglik_grad")
            ctx.save_for_backward(dpri, dchan.to(chan.device))
        else:
            st = batch.loglik_into(rx, pr, ll)
            if st != 0:
                raise mapdec.MapDecError(st, "mapdec_batch_decode")
        ctx.sym_off = batch.sym_off.copy()
        ctx.sizes = [f.N * f.q for f in batch.frames]
        ctx.dtypes = (priors_all.dtype, chan.dtype)
        return ll

    @staticmethod
    def backward(ctx, grad_out):
        dpri, dchan = ctx.saved_tensors
        g = grad_out.to(torch.float64)
        gp = None
        if ctx.needs_input_grad[0]:
            scale = torch.empty(dpri.numel(), dtype=torch.float64, device=dpri.device)
            gd = g.to(dpri.device)
            for k, (o, sz) in enumerate(zip(ctx.sym_off, ctx.sizes)):
                scale[int(o):int(o) + sz] = gd[k]
            gp = (dpri.to(torch.float64) * scale).to(ctx.dtypes[0])
        gc = (dchan * g.to(dchan.device)[:, None]).to(ctx.dtypes[1]) \
            if ctx.needs_input_grad[1] else None
        return gp, gc, None, None


def frame_loglik(priors, chan, decoder, rx):
    return FrameLogLik.apply(priors, chan, decoder, rx)


def batch_loglik(priors_all, chan, batch, rx_all):
    return BatchLogLik.apply(priors_all, chan, batch, rx_all)
