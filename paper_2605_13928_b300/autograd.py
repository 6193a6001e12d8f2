"""KL(P || Q) of t-SNE as a torch.autograd.Function over the CUDA kernels.

KLDivergence.apply(Y, P, alpha, batch) returns KL_alpha(Y) summed over the
samples, with

    KL_alpha = sum p log p + alpha sum p log(1 + |y_i - y_j|^2) + log Z,

which is KL(P || Q) at alpha = 1 (van der Maaten & Hinton 2008, Eq. 2 with
Q of Eq. 4) and whose gradient is the exaggerated t-SNE gradient
4 sum_j (alpha p_ij - q_ij) w_ij (y_i - y_j) (their Eq. 5).  Z needs the full
O(n^2) sweep, which yields the repulsive forces at no extra cost, so the
forward pass runs tsne_kl_grad once for both the value and the gradient; the
backward pass scales the saved gradient by the incoming gradient.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import _lib as L
from . import api


class KLDivergence(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Y: torch.Tensor, P: api.CSR, alpha: float = 1.0,
                batch: Optional[api.Batch] = None, params: Optional[L.TsneParams] = None,
                ws: Optional[api.Workspace] = None):
        need_grad = ctx.needs_input_grad[0]
        Yc = Y.detach().contiguous()
        g, Z, kl = api.kl_grad(P, Yc, alpha, batch=batch, want_grad=need_grad, want_kl=True,
                               params=params, ws=ws)
        if need_grad:
            ctx.save_for_backward(g)
        return kl.sum()

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return g * grad_out.to(g.dtype), None, None, None, None, None


def kl_divergence(Y: torch.Tensor, P: api.CSR, alpha: float = 1.0,
                  batch: Optional[api.Batch] = None, params: Optional[L.TsneParams] = None,
                  ws: Optional[api.Workspace] = None) -> torch.Tensor:
    """KL_alpha(Y) (float64 scalar) with the exact gradient w.r.t. Y (float32)."""
    return KLDivergence.apply(Y, P, alpha, batch, params, ws)
