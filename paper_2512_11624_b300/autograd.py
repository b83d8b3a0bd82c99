"""torch.autograd.Function front ends over the library's forward and adjoint.

Both functions hold a `gsvr.Context` (stacks, observations and the current
pixel sample live in it) and pass parameters and gradients as CUDA tensors in
the library's parameter-vector layout (11 N Gaussian entries, then 6 per slice).

- `SliceLoss.apply(theta, gs)` returns the MSE loss of the sampled pixels
  (Eq. 5 numerator with the exact-convolution normalisation, the slice model of
  Eq. 1 / 3 / 4); its backward scales the library's dL/dtheta by the incoming
  gradient.
- `SlicePredict.apply(theta, gs)` returns the predicted intensities of the
  sampled pixels (in the library's sample order, `gs.sample_index()`); its
  backward writes the incoming dL/dI_hat into the library's per-pixel adjoint
  buffer and runs the same tile adjoint, so any downstream loss differentiates
  through the analytic-PSF model.

Neither stores anything per (pixel, Gaussian) pair: the backward recomputes each
pair from the sorted tile lists of the forward, including the slice-pose
gradients.  The forward of the context must not change between a function's
forward and its backward (the tile lists are the context's).
"""
from __future__ import annotations

import torch

from . import gsvr


def _load(gs, theta):
    if theta.device != gs.theta.device or theta.dtype != torch.float32 or theta.numel() != gs.n_params:
        raise ValueError("theta must be a float32 CUDA tensor of %d entries on %s" % (gs.n_params, gs.theta.device))
    gs.theta.copy_(theta.detach().reshape(-1))


class SliceLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, gs):
        _load(gs, theta)
        gsvr.gsvr_forward(gs.ctx)
        ctx.gs = gs
        return gs.loss_t.clone().reshape(())

    @staticmethod
    def backward(ctx, grad_loss):
        gs = ctx.gs
        gsvr.gsvr_backward(gs.ctx)
        g = gs.grad.clone() * grad_loss.to(torch.float32)
        return g, None


class SlicePredict(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, gs):
        _load(gs, theta)
        gsvr.gsvr_forward(gs.ctx)
        idx = gs.sample_index()
        ctx.gs = gs
        ctx.idx = idx
        return gs.pred.index_select(0, idx)

    @staticmethod
    def backward(ctx, grad_pred):
        gs = ctx.gs
        gs.rbar.index_copy_(0, ctx.idx, grad_pred.to(torch.float32).contiguous())
        gsvr.gsvr_backward(gs.ctx)
        return gs.grad.clone(), None


def recompute_vs_store_bytes(gs):
    """Device bytes of the adjoint's intermediate state per step: what this
    library keeps (tile-ordered records, keys, per-key moments) against what a
    store-per-pair adjoint would keep (one float32 factor per evaluated
    (pixel, Gaussian) pair)."""
    st = gs.stats()
    kept = st["n_keys"] * (32 + 32 + 4 + 4) + st["n_records"] * (32 + 8 + 4 + 4)
    stored = st["pairs_evaluated"] * 4
    return {"recompute_bytes": int(kept), "store_per_pair_bytes": int(stored),
            "pairs_evaluated": st["pairs_evaluated"], "keys": st["n_keys"], "records": st["n_records"]}
