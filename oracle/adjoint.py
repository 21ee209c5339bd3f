"""Gradients through X = P^{-1} F, in FP64 on the CPU (test infrastructure).

Not in the paper.  For a loss L(X) with G = dL/dX, the adjoint identity gives
lambda = P^{-T} G, dL/dF = lambda and dL/dP = -lambda X^T.  P holds -A_j,
C_j and -B_j (eq. main-eq), hence, summed over the K right-hand sides,

    dL/dC_j = -lambda_j X_j^T,  dL/dA_j = lambda_j X_{j-1}^T (j > 1),
    dL/dB_j = lambda_j X_{j+1}^T (j < N),  dL/dA_1 = dL/dB_N = 0.

P^T is block tridiagonal again: A'_j = B_{j-1}^T, B'_j = A_{j+1}^T, C'_j = C_j^T.
"""

from __future__ import annotations

import numpy as np

from .blocktri import solve_block_thomas


def transpose_blocks(A, B, C):
    """Blocks of P^T in the layout of eq. main-eq."""
    N, M, _ = C.shape
    At = np.zeros_like(A)
    Bt = np.zeros_like(B)
    At[1:] = np.transpose(B[:-1], (0, 2, 1))
    Bt[:-1] = np.transpose(A[1:], (0, 2, 1))
    Ct = np.transpose(C, (0, 2, 1)).copy()
    return At, Bt, Ct


def adjoint_grads(A, B, C, X, G):
    """(dF, dA, dB, dC) for upstream gradient G = dL/dX at the solution X."""
    lam = solve_block_thomas(*transpose_blocks(A, B, C), G)
    dC = -np.einsum("jak,jbk->jab", lam, X)
    dA = np.zeros_like(A)
    dB = np.zeros_like(B)
    dA[1:] = np.einsum("jak,jbk->jab", lam[1:], X[:-1])
    dB[:-1] = np.einsum("jak,jbk->jab", lam[:-1], X[1:])
    return lam, dA, dB, dC
