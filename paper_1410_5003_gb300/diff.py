"""Differentiable solve of the reduced block-tridiagonal system A' eta = f
(Sec. 3.3) for torch autograd: the forward pass uses the block factors of a
context's last FP64 solve (mlqp_solve_rhs), the backward pass the transposed
block sweep with the same factors (mlqp_adjoint_solve).  For the real loss
L(eta), torch's complex gradient convention gives dL/df = A'^{-H} dL/deta."""
import torch


class BlockSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, f, ctx):
        fctx.mlqp_ctx = ctx
        return ctx.solve_rhs(f)

    @staticmethod
    def backward(fctx, grad_eta):
        return fctx.mlqp_ctx.adjoint_solve(grad_eta), None


def block_solve(ctx, f):
    """eta = A'^{-1} f, differentiable in f (ctx: a Context after an FP64 solve)."""
    return BlockSolve.apply(f, ctx)
