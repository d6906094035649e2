"""torch.autograd.Function wrappers of the libcgs forward/backward.

The backward never stores per-pixel splat lists: it recomputes transmittance from
the stored final T and last-contributor index (cgs_raster_bwd), then applies the
chain rule to the parameters (cgs_preprocess_bwd).

  * RasterizeWindow: params -> per-view loss L_v (L1 photometric + depth, fused in
    the forward kernel).  Backward scales each view's pixel gradients by the
    incoming dL/dL_v.
  * RenderWindow: params -> (images, depths) for a caller-defined loss; backward
    takes dL/dimage and dL/ddepth from autograd.

Both use a MappingWindow as the holder of cameras, targets and work buffers.
"""
from __future__ import annotations

import torch

from .window import MappingWindow


class RasterizeWindow(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, win: MappingWindow):
        p = params.detach().contiguous()
        win.forward(with_loss=True, params=p)
        ctx.win = win
        ctx.save_for_backward(p)
        return win.loss_view.clone()

    @staticmethod
    def backward(ctx, grad_loss: torch.Tensor):
        win: MappingWindow = ctx.win
        (p,) = ctx.saved_tensors
        base = win.view_weight.clone()
        win.view_weight.mul_(grad_loss.contiguous())
        grads = torch.empty_like(p)
        try:
            win.backward(params=p, grads_out=grads)
        finally:
            win.view_weight.copy_(base)
        return grads, None


class RenderWindow(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, win: MappingWindow):
        p = params.detach().contiguous()
        win.forward(with_loss=False, params=p)
        ctx.win = win
        ctx.save_for_backward(p)
        return win.img.clone(), win.depth.clone()

    @staticmethod
    def backward(ctx, g_img: torch.Tensor, g_depth: torch.Tensor):
        win: MappingWindow = ctx.win
        (p,) = ctx.saved_tensors
        gi = torch.zeros_like(win.img) if g_img is None else g_img.contiguous()
        gd = None if g_depth is None else g_depth.contiguous()
        grads = torch.empty_like(p)
        win.backward(dl_dimg=gi, dl_ddepth=gd, params=p, grads_out=grads)
        return grads, None
