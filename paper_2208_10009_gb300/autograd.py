"""torch.autograd.Function over the fixed-face-sequence unfolding (forward and adjoint
CUDA kernels of the library).  Backward recomputes the unfolding from the saved inputs;
no per-bounce state is stored."""
from __future__ import annotations

import torch

from .api import Context, Scene


class SbrUnfold(torch.autograd.Function):
    """outputs (P, 8) = (miss xyz, delay, AOD az, AOD el, AOA az, AOA el) of paths given by
    tx (P, 3), rx (P, 3), az_el (P, 2) and fixed faces (P, 8) int32 / order (P,) int32."""

    @staticmethod
    def forward(ctx, lib: Context, scene: Scene, tx, rx, az_el, faces, order):
        tx, rx, az_el = tx.contiguous().float(), rx.contiguous().float(), az_el.contiguous().float()
        faces, order = faces.contiguous().int(), order.contiguous().int()
        out = lib.unfold_fwd(scene, tx, rx, az_el, faces, order)
        ctx.save_for_backward(tx, rx, az_el, faces, order)
        ctx.lib, ctx.scene = lib, scene
        return out

    @staticmethod
    def backward(ctx, grad_out):
        tx, rx, az_el, faces, order = ctx.saved_tensors
        g_tx, g_rx, g_ae = ctx.lib.unfold_bwd(ctx.scene, tx, rx, az_el, faces, order, grad_out.contiguous().float())
        return None, None, g_tx, g_rx, g_ae, None, None


def unfold(lib: Context, scene: Scene, tx, rx, az_el, faces, order):
    return SbrUnfold.apply(lib, scene, tx, rx, az_el, faces, order)
