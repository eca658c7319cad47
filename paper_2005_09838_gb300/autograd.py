"""torch.autograd face of the differentiation form (tc_grad_* in the C ABI).

``factor_loss(X, Y, g)`` is the loss of the factor model,
L(X, Y) = 1/2 ||P_Omega(X*Y - G)||_F^2 + rho1/2 ||H unfold(X*Y, 1)||_F^2,
for spatial CUDA tensors X of shape (n1, r, n3) and Y of shape (r, n2, n3); the
forward pass runs the library's loss and adjoint kernels (one call gives the
loss and both gradients), the backward pass scales the stored gradients.
This module only moves tensors between the (i1, s, i3) indexing and the
column-major layout of the C ABI.

``block_gradient_descent`` alternates gradient steps on the X and Y blocks
(the block scheme of Eq. (updataXYW1) with plain gradient directions).
"""
from __future__ import annotations

import torch

from . import tc


def _colmajor(t: torch.Tensor) -> torch.Tensor:
    return t.detach().permute(2, 1, 0).contiguous()


def grad_context(G, mask, r: int, rho1: float = 0.0, dtype=torch.float32, stream: int | None = None):
    """GradContext for observed data G (n1, n2, n3) and boolean mask, as CUDA
    tensors or numpy arrays."""
    G = torch.as_tensor(G)
    mask = torch.as_tensor(mask)
    n1, n2, n3 = G.shape
    prec = tc.TC_FP64 if dtype == torch.float64 else tc.TC_FP32
    p = tc.make_params(n1, n2, n3, r, rho1=rho1, precision=prec)
    g = _colmajor(G.to(device="cuda", dtype=dtype))
    m = _colmajor(mask.to(device="cuda", dtype=torch.uint8))
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    ctx = tc.GradContext(p, g, m, on_device=True, stream=stream)
    torch.cuda.current_stream().synchronize()
    return ctx


class FactorLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, Y, g):
        Xc, Yc = _colmajor(X), _colmajor(Y)
        dXc, dYc = torch.empty_like(Xc), torch.empty_like(Yc)
        loss = g.eval(Xc, Yc, dXc, dYc, on_device=True)
        ctx.save_for_backward(dXc.permute(2, 1, 0), dYc.permute(2, 1, 0))
        return torch.tensor(loss, dtype=X.dtype, device=X.device)

    @staticmethod
    def backward(ctx, g_loss):
        dX, dY = ctx.saved_tensors
        return g_loss * dX, g_loss * dY, None


def factor_loss(X: torch.Tensor, Y: torch.Tensor, g) -> torch.Tensor:
    return FactorLoss.apply(X, Y, g)


def block_gradient_descent(g, X: torch.Tensor, Y: torch.Tensor, steps: int, lr_x: float, lr_y: float,
                           max_halvings: int = 30):
    """Alternate X <- X - t_x dL/dX (Y fixed) and Y <- Y - t_y dL/dY (new X).
    The block Lipschitz constants change with the other block, so each step
    starts from lr and halves it until the loss decreases (backtracking on the
    library's loss).  Returns the final factors and the loss after every
    accepted block step (strictly decreasing)."""
    X = X.detach().clone().requires_grad_(True)
    Y = Y.detach().clone().requires_grad_(True)
    with torch.no_grad():
        hist = [float(factor_loss(X, Y, g))]
    for _ in range(steps):
        for block, lr0 in ((X, lr_x), (Y, lr_y)):
            X.grad = None
            Y.grad = None
            loss = factor_loss(X, Y, g)
            loss.backward()
            f0 = float(loss.detach())
            step = block.grad.detach().clone()
            lr = lr0
            with torch.no_grad():
                for _ in range(max_halvings):
                    block.sub_(lr * step)
                    try:
                        f1 = float(factor_loss(X, Y, g))
                    except tc.TCError:
                        f1 = float("inf")
                    if f1 < f0:
                        break
                    block.add_(lr * step)
                    lr *= 0.5
                else:
                    f1 = f0
            hist.append(f1)
    return X.detach(), Y.detach(), hist
