"""Band matrices as block-tridiagonal systems, in FP64 on the CPU (test infrastructure).

Section 3.3.1, item c: the PML operator A_44 is a band matrix that the
dichotomy algorithm solves as a block-tridiagonal matrix whose off-diagonal
blocks are triangular.  Written out by definition here:

* the band matrix Q of order n with kl sub- and ku super-diagonals, from the
  diagonal-ordered storage ab[ku + i - j, j] = Q[i, j] (the layout of LAPACK's
  general band routines and SciPy's banded solver);
* its cut into N = S ceil(ceil(n / M) / S) block rows of M rows, padded with
  the identity beyond order n, in the sign convention of eq. main-eq:
  C_j = Q[jM.., jM..], A_j = -Q[jM.., (j-1)M..], B_j = -Q[jM.., (j+1)M..].
"""

from __future__ import annotations

import numpy as np


def band_dense(ab, kl: int, ku: int):
    """The dense n x n matrix Q held in diagonal-ordered storage ab [kl + ku + 1, n]."""
    n = ab.shape[1]
    Q = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            Q[i, j] = ab[ku + i - j, j]
    return Q


def band_blocks(ab, kl: int, ku: int, M: int, S: int):
    """(A, B, C, N): the block-tridiagonal form of Q with M x M blocks and N
    block rows (a multiple of S), identity-padded beyond order n."""
    n = ab.shape[1]
    N = -(-(-(-n // M)) // S) * S
    Qp = np.eye(N * M)
    Qp[:n, :n] = band_dense(ab, kl, ku)
    A = np.zeros((N, M, M))
    B = np.zeros((N, M, M))
    C = np.zeros((N, M, M))
    for j in range(N):
        r = slice(j * M, (j + 1) * M)
        C[j] = Qp[r, r]
        if j > 0:
            A[j] = -Qp[r, (j - 1) * M:j * M]
        if j < N - 1:
            B[j] = -Qp[r, (j + 1) * M:(j + 2) * M]
    return A, B, C, N


def pad_rows(F, N: int, M: int):
    """The [N, M, K] panel of an n x K right-hand side, zero beyond row n."""
    n, K = F.shape
    Fp = np.zeros((N * M, K))
    Fp[:n] = F
    return Fp.reshape(N, M, K)
