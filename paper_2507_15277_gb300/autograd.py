"""torch.autograd.Function for Y = X @ W on the portability-tuned SGEMM.

Forward is one pt_sgemm call (NN).  Backward computes
    dX = G @ W^T   (pt_sgemm with transB = 'T', an NT problem)
    dW = X^T @ G   (pt_sgemm with transA = 'T', a TN problem)
through the same runtime selector, so tuned NT/TN shapes in the loaded
manifest are used for the gradients.  Every product runs in the library's
kernels; torch only provides the tensors and the autograd graph.
"""

from __future__ import annotations

import torch

from . import sgemm


def _rowmajor(t):
    return t if (t.dim() == 2 and (t.shape[1] <= 1 or t.stride(1) == 1)) else t.contiguous()


class SgemmFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, W):
        if X.dtype != torch.float32 or W.dtype != torch.float32:
            raise TypeError("float32 only")
        X = _rowmajor(X)
        W = _rowmajor(W)
        ctx.save_for_backward(X, W)
        return sgemm(X, W)

    @staticmethod
    def backward(ctx, G):
        X, W = ctx.saved_tensors
        G = _rowmajor(G)
        dX = dW = None
        if ctx.needs_input_grad[0]:
            dX = sgemm(G, W, transB="T")
        if ctx.needs_input_grad[1]:
            dW = sgemm(X, G, transA="T")
        return dX, dW


def matmul(X, W):
    """Y = X @ W with gradients through the tuned SGEMM."""
    return SgemmFunction.apply(X, W)
