"""The block-tridiagonal system by definition, in FP64 on the CPU (test infrastructure).

System (Section 2, eq. main-eq), block row j = 1..N (index j-1 here):

    -A_j X_{j-1} + C_j X_j - B_j X_{j+1} = F_j,     A_j, B_j, C_j in R^{M x M},

with no A term in the first row and no B term in the last (the matrix shape
printed with eq. main-eq).  X and F are [N, M, K] panels: K right-hand sides
against the same matrix (abstract; Algorithm 2's split into a preliminary stage
and a per-right-hand-side stage).

The method of the paper is a direct solver: in exact arithmetic it returns
X = P^{-1} F.  The oracle is therefore that definition written out -- block
Gaussian elimination without block interchanges (block Thomas, the matrix sweep
the paper cites for its pre-factorised segment solves), with each pivot block
solved by LAPACK's partially pivoted LU, and dense LU of the assembled matrix
for tiny systems.
"""

from __future__ import annotations

import numpy as np


def apply_P(A, B, C, X):
    """Y = P X for the operator of eq. main-eq; A[0] and B[N-1] are ignored."""
    Y = np.einsum("jab,jbk->jak", C, X)
    Y[1:] -= np.einsum("jab,jbk->jak", A[1:], X[:-1])
    Y[:-1] -= np.einsum("jab,jbk->jak", B[:-1], X[1:])
    return Y


def dense_P(A, B, C):
    """The assembled (N*M) x (N*M) matrix of eq. main-eq."""
    N, M, _ = C.shape
    P = np.zeros((N * M, N * M))
    for j in range(N):
        r = slice(j * M, (j + 1) * M)
        P[r, r] = C[j]
        if j > 0:
            P[r, (j - 1) * M:j * M] = -A[j]
        if j < N - 1:
            P[r, (j + 1) * M:(j + 2) * M] = -B[j]
    return P


def solve_dense(A, B, C, F):
    """X = P^{-1} F by dense LU (LAPACK gesv) of the assembled matrix; tiny systems only."""
    N, M, K = F.shape
    X = np.linalg.solve(dense_P(A, B, C), F.reshape(N * M, K))
    return X.reshape(N, M, K)


def solve_block_thomas(A, B, C, F):
    """X = P^{-1} F by block Gaussian elimination (matrix sweep).

    Forward:  D_1 = C_1;  D_j = C_j - A_j alpha_{j-1};  alpha_j = D_j^{-1} B_j;
              beta_j = D_j^{-1} (F_j + A_j beta_{j-1})
    Backward: X_N = beta_N;  X_j = beta_j + alpha_j X_{j+1}.
    Each D_j^{-1} [B_j | rhs] is one LAPACK solve with partial pivoting.
    """
    N, M, K = F.shape
    alpha = np.empty((N, M, M))
    beta = np.empty((N, M, K))
    prev_alpha = None
    prev_beta = None
    for j in range(N):
        if j == 0:
            D = C[0]
            rhs_F = F[0]
        else:
            D = C[j] - A[j] @ prev_alpha
            rhs_F = F[j] + A[j] @ prev_beta
        sol = np.linalg.solve(D, np.concatenate([B[j], rhs_F], axis=1))
        alpha[j] = sol[:, :M]
        beta[j] = sol[:, M:]
        prev_alpha, prev_beta = alpha[j], beta[j]
    X = np.empty_like(beta)
    X[N - 1] = beta[N - 1]
    for j in range(N - 2, -1, -1):
        X[j] = beta[j] + alpha[j] @ X[j + 1]
    return X


def residual(A, B, C, X, F):
    """r = F - P X."""
    return F - apply_P(A, B, C, X)


def rel_err(X, X_ref):
    """||X - X_ref||_F / ||X_ref||_F over the whole panel."""
    return float(np.linalg.norm((X - X_ref).ravel()) / np.linalg.norm(X_ref.ravel()))


def col_err(X, X_ref):
    """max over right-hand-side columns n of max_i |X - X_ref|[i, n] / max_i |X_ref|[i, n],
    i running over the N*M rows of the panel (each column measured on its own); a
    1-D vector is one column."""
    K = X.shape[-1] if X.ndim > 1 else 1
    D = np.abs(X - X_ref).reshape(-1, K).max(axis=0)
    R = np.abs(X_ref).reshape(-1, K).max(axis=0)
    return float(np.max(D / R))


def rel_res(A, B, C, X, F):
    """||F - P X||_F / ||F||_F over the whole panel."""
    return float(np.linalg.norm(residual(A, B, C, X, F).ravel()) / np.linalg.norm(F.ravel()))
