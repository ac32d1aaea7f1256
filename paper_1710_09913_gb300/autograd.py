"""torch.autograd.Function wrappers around the DoGIP kernels.

* ``dogip_apply(u, op)``: y = K u; backward: grad_u = K grad_y (K is symmetric).
* ``dogip_solve(A, b, op)``: u = K(A)^-1 b with K(A) the DoGIP operator of the
  coefficients A (per-element scalars [E] or symmetric tensors [E, d, d]);
  backward: adjoint solve K lambda = grad_u (K symmetric), grad_b = lambda and
  grad_A = -(dK/dA)[lambda, u], evaluated per element on the W nodes as
  -sum_j om_j (grad lambda)(x_j) (x) (grad u)(x_j) (om_j = |det R_T| w_j): the
  per-node outer product that the element-wise DoGIP factorisation (eq.
  ep_dogip_mul / wp_dogip_mul with the coefficient factored out) makes cheap.
  Gradients at the W nodes are recomputed from u and lambda, never stored.
  K depends on the symmetric part of each tensor, so the tensor gradient is
  symmetrised.

Everything runs in the CUDA library; these classes only route tensors.  The
operator ``op`` (a ``binding.Context``) keeps the coefficients of the last
forward call.
"""

from __future__ import annotations

import torch

from . import binding


class DogipApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, op, prec):
        ctx.op, ctx.prec = op, prec
        return op.apply(u.contiguous(), prec=prec)

    @staticmethod
    def backward(ctx, gy):
        return ctx.op.apply(gy.contiguous(), prec=ctx.prec), None, None


class DogipSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, b, op, solve_kwargs):
        A64 = A.detach().to(torch.float64).contiguous()
        op.set_coef(A64)
        u, info = op.solve(b.detach().to(torch.float64).contiguous(), **solve_kwargs)
        ctx.op, ctx.kw, ctx.A_dtype, ctx.A_shape = op, solve_kwargs, A.dtype, A.shape
        ctx.save_for_backward(A64, u)
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, gu):
        A64, u = ctx.saved_tensors
        op = ctx.op
        op.set_coef(A64)  # the operator may have been reused since forward
        lam, _ = op.solve(gu.detach().to(torch.float64).contiguous(), **ctx.kw)
        gA = op.grad_coef(u, lam)
        if gA.dim() == 3:
            gA = 0.5 * (gA + gA.transpose(1, 2))
        return gA.to(ctx.A_dtype).reshape(ctx.A_shape), lam, None, None


def dogip_apply(u: torch.Tensor, op: "binding.Context", prec: str = "fp64") -> torch.Tensor:
    return DogipApply.apply(u, op, prec)


def dogip_solve(A: torch.Tensor, b: torch.Tensor, op: "binding.Context", **solve_kwargs) -> torch.Tensor:
    return DogipSolve.apply(A, b, op, solve_kwargs)


def compliance(A: torch.Tensor, b: torch.Tensor, op: "binding.Context", **solve_kwargs) -> torch.Tensor:
    """J(A) = b^T u(A) with K(A) u = b (differentiable in A)."""
    return torch.dot(b.to(torch.float64), dogip_solve(A, b, op, **solve_kwargs))
