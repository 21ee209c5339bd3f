"""torch.autograd.Function around the block-tridiagonal solve.

Forward: factor P from (A, B, C) (Algorithm 2, stage 1) and solve X = P^{-1} F
(stage 2).  Backward: bt_solve_adjoint solves P^T lambda = dL/dX with the factors
of P^T and returns dL/dF = lambda and the block gradients
dL/dC_j = -lambda_j X_j^T, dL/dA_j = lambda_j X_{j-1}^T, dL/dB_j = lambda_j X_{j+1}^T.
All arithmetic runs in libbt's kernels; this module only moves tensors.

Inputs of any floating dtype are accepted; the factors and the adjoint are
always FP64, the forward solve runs in the requested precision and the outputs
and gradients are returned in the dtype of the corresponding input.
"""

from __future__ import annotations

import torch

from .solver import factor


class BTSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, C, F, S: int, precision: str = "f64", tol: float = 0.0):
        fac = factor(A.detach().double().contiguous(), B.detach().double().contiguous(),
                     C.detach().double().contiguous(), S)
        X = fac.solve(F.detach().double().contiguous(), precision=precision, tol=tol)
        ctx.fac = fac
        ctx.dtypes = (A.dtype, B.dtype, C.dtype, F.dtype)
        ctx.save_for_backward(X)
        return X.to(F.dtype)

    @staticmethod
    def backward(ctx, gX):
        (X,) = ctx.saved_tensors
        want = tuple(n for n, need in zip("ABCF", ctx.needs_input_grad[:4]) if need)
        dF, dA, dB, dC = ctx.fac.adjoint(X, gX.double().contiguous(), want=want)
        tA, tB, tC, tF = ctx.dtypes
        out = (dA.to(tA) if dA is not None else None, dB.to(tB) if dB is not None else None,
               dC.to(tC) if dC is not None else None, dF.to(tF) if dF is not None else None)
        ctx.fac.close()
        ctx.fac = None
        return out + (None, None, None)


def bt_solve(A, B, C, F, S: int, precision: str = "f64", tol: float = 0.0):
    """Differentiable X = P^{-1} F for blocks A, B, C [N, M, M] and panel F [N, M, K]."""
    return BTSolve.apply(A, B, C, F, S, precision, tol)
