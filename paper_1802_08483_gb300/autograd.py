"""torch.autograd.Function wrappers around the decoder's adjoint path.

forward() calls mapdec_loglik_grad / mapdec_batch_loglik_grad (the CUDA
kernels compute log P(Y) together with d logP / d(Pi, Pd, Ps) and
d logP / d prior) and saves the gradients; backward() scales them by the
incoming gradient.  PyTorch only moves the tensors; every step of the
computation runs in libmapdec.so.
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


class FrameLogLik(torch.autograd.Function):
    """log P(Y) of one frame as a function of (priors (N, q), chan = [Pi, Pd, Ps]).

    The decoder handle carries the code and channel; chan must hold the same
    channel values the handle was created with (the derivative is taken there).
    """

    @staticmethod
    def forward(ctx, priors, chan, decoder, rx):
        if not _same_channel(_chan_tuple(chan), (decoder.Pi, decoder.Pd, decoder.Ps)):
            raise ValueError("chan differs from the decoder's channel parameters")
        pr = priors.detach().to("cpu", torch.float32).contiguous().numpy()
        ll, dchan, dpri = decoder.loglik_grad(np.asarray(rx, np.uint8), pr)
        ctx.save_for_backward(torch.from_numpy(np.asarray(dpri, np.float32)).to(priors.device),
                              torch.from_numpy(np.asarray(dchan, np.float64)).to(chan.device))
        ctx.dtypes = (priors.dtype, chan.dtype)
        return torch.tensor(ll, dtype=torch.float64, device=priors.device)

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
        st, dchan, dpri, ll = batch.loglik_grad(np.asarray(rx_all, np.uint8),
                                                priors_all.detach().to("cpu", torch.float32)
                                                .contiguous().numpy())
        if st != 0:
            raise mapdec.MapDecError(st, "mapdec_batch_loglik_grad")
        ctx.save_for_backward(torch.from_numpy(dpri).to(priors_all.device),
                              torch.from_numpy(dchan).to(chan.device))
        ctx.sym_off = batch.sym_off.copy()
        ctx.sizes = [f.N * f.q for f in batch.frames]
        ctx.dtypes = (priors_all.dtype, chan.dtype)
        return torch.from_numpy(ll).to(priors_all.device)

    @staticmethod
    def backward(ctx, grad_out):
        dpri, dchan = ctx.saved_tensors
        g = grad_out.to(torch.float64)
        gp = None
        if ctx.needs_input_grad[0]:
            scale = torch.empty(dpri.numel(), dtype=torch.float64, device=dpri.device)
            for k, (o, sz) in enumerate(zip(ctx.sym_off, ctx.sizes)):
                scale[int(o):int(o) + sz] = g[k]
            gp = (dpri.to(torch.float64) * scale).to(ctx.dtypes[0])
        gc = (dchan * g.to(dchan.device)[:, None]).to(ctx.dtypes[1]) \
            if ctx.needs_input_grad[1] else None
        return gp, gc, None, None


def frame_loglik(priors, chan, decoder, rx):
    return FrameLogLik.apply(priors, chan, decoder, rx)


def batch_loglik(priors_all, chan, batch, rx_all):
    return BatchLogLik.apply(priors_all, chan, batch, rx_all)
