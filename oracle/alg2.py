"""Segment / interface decomposition of Section 2.2, written out by definition (test infrastructure).

Rows are 0-based here: paper row i is index i-1.  With S segments of L = N/S rows,
segment s owns rows [k_s, k_s + L) with interface row k_s = s*L (the paper's
K = 1, L+1, ..., (p-1)L+1) and interior rows k_s+1 .. k_s+L-1; the row after the
last segment is the fictitious X_{N+1} = 0 (eq. superposition).

* ``segment_responses`` -- U, V of eqs. sub1 / sub2: the interior solution with
  unit data at the left / right end of the segment and zero right-hand side.
* ``segment_W``          -- W of eq. sub3: the interior solution with the true
  right-hand side and zero ends.
* ``reduced_system``     -- the blocks of eq. red1 (the reduced matrix P~).
* ``reduced_rhs``        -- its right-hand side F~.
* ``dichotomy_tree`` / ``dichotomy_solve`` -- Algorithm 1 applied to P~: the
  middle unknown of every subsystem from the stored block row of the
  subsystem's inverse, then the two halves with the end blocks of their
  right-hand sides modified by the computed unknown (eqs. suba / subb).
* ``alg2_solve``         -- Algorithm 2, stage 2: W, then P~ X~ = F~ by the
  dichotomy, then every row from eq. superposition.

Every subsystem here is solved by dense LU of its assembled matrix, i.e. by
its definition; nothing is blocked, fused or reordered.
"""

from __future__ import annotations

import dataclasses
from typing import List, Tuple

import numpy as np

from .blocktri import dense_P


def segment_rows(N: int, S: int) -> List[Tuple[int, int, int]]:
    """[(k_s, first interior row, one past the last interior row)] for s = 0..S-1."""
    if S < 1 or N % S != 0:
        raise ValueError("the segment count must divide N (L = N/p)")
    L = N // S
    return [(s * L, s * L + 1, s * L + L) for s in range(S)]


def _interior_matrix(A, B, C, a, b):
    """Assembled matrix of rows a..b-1 with the couplings outside the range dropped."""
    return dense_P(A[a:b].copy(), B[a:b].copy(), C[a:b].copy())


def segment_responses(A, B, C, S):
    """U, V ([N, M, M]; zero on interface rows) from eqs. sub1 and sub2."""
    N, M, _ = C.shape
    U = np.zeros((N, M, M))
    V = np.zeros((N, M, M))
    for k, a, b in segment_rows(N, S):
        n = b - a
        if n == 0:
            continue
        P = _interior_matrix(A, B, C, a, b)
        rhs_u = np.zeros((n * M, M))
        rhs_v = np.zeros((n * M, M))
        # -A_a U_{a-1} with U_k = I moves to the right-hand side as +A_a.
        rhs_u[:M] = A[a]
        # -B_{b-1} V_b with V_{k+L} = I moves to the right-hand side as +B_{b-1};
        # the last row of the system has no B (X_{N+1} = 0), stored as zero.
        rhs_v[(n - 1) * M:] = B[b - 1] if b - 1 < N - 1 else 0.0
        U[a:b] = np.linalg.solve(P, rhs_u).reshape(n, M, M)
        V[a:b] = np.linalg.solve(P, rhs_v).reshape(n, M, M)
    return U, V


def segment_W(A, B, C, F, S):
    """W ([N, M, K]; zero on interface rows) from eq. sub3."""
    N, M, K = F.shape
    W = np.zeros((N, M, K))
    for k, a, b in segment_rows(N, S):
        n = b - a
        if n == 0:
            continue
        P = _interior_matrix(A, B, C, a, b)
        W[a:b] = np.linalg.solve(P, F[a:b].reshape(n * M, K)).reshape(n, M, K)
    return W


def _neighbour_responses(U, V, N, S, M):
    """Superposition coefficients of the rows next to every interface.

    Row k_s - 1 is written in segment s-1's representation and row k_s + 1 in
    segment s's.  With L = 1 those rows are interfaces themselves: X_{k-1} is
    X~_{s-1} (U = I, V = 0) and X_{k+1} is X~_{s+1} (U = 0, V = I); this makes
    P~ = P when every row is an interface.
    """
    L = N // S
    I = np.eye(M)
    Z = np.zeros((M, M))
    left = []   # (U_{K-1}, V_{K-1}) per interface
    right = []  # (U_{K+1}, V_{K+1}) per interface
    for s in range(S):
        K = s * L
        if s == 0:
            left.append((Z, Z))
        elif L == 1:
            left.append((I, Z))
        else:
            left.append((U[K - 1], V[K - 1]))
        if K + 1 >= N:
            right.append((Z, Z))
        elif L == 1:
            right.append((Z, I))
        else:
            right.append((U[K + 1], V[K + 1]))
    return left, right


def reduced_system(A, B, C, S, U, V):
    """Blocks (At, Ct, Bt), each [S, M, M], of eq. red1:
    -At_s X~_{s-1} + Ct_s X~_s - Bt_s X~_{s+1} = F~_s with
    At_s = A_K U_{K-1},  Ct_s = C_K - A_K V_{K-1} - B_K U_{K+1},  Bt_s = B_K V_{K+1},
    K = k_s and U_0 = V_0 = 0."""
    N, M, _ = C.shape
    L = N // S
    left, right = _neighbour_responses(U, V, N, S, M)
    At = np.zeros((S, M, M))
    Ct = np.zeros((S, M, M))
    Bt = np.zeros((S, M, M))
    for s in range(S):
        K = s * L
        Ul, Vl = left[s]
        Ur, Vr = right[s]
        Ak = A[K] if K > 0 else np.zeros((M, M))
        Bk = B[K] if K < N - 1 else np.zeros((M, M))
        At[s] = Ak @ Ul
        Ct[s] = C[K] - Ak @ Vl - Bk @ Ur
        Bt[s] = Bk @ Vr
    return At, Ct, Bt


def reduced_rhs(A, B, F, W, S):
    """F~_s = F_K + A_K W_{K-1} + B_K W_{K+1} (eq. red1); W is zero on interface rows."""
    N, M, K_ = F.shape
    L = N // S
    Ft = np.zeros((S, M, K_))
    for s in range(S):
        K = s * L
        Ft[s] = F[K]
        if K > 0:
            Ft[s] += A[K] @ W[K - 1]
        if K < N - 1:
            Ft[s] += B[K] @ W[K + 1]
    return Ft


@dataclasses.dataclass
class Node:
    l: int
    r: int
    m: int
    level: int
    R: np.ndarray   # [r-l+1, M, M]: block row m of ({P~}_l^r)^{-1}, columns l..r
    HL: np.ndarray  # R_{m,l} At_l   (zero if l == 0)
    HR: np.ndarray  # R_{m,r} Bt_r   (zero if r == S-1)


def dichotomy_tree(At, Ct, Bt) -> List[Node]:
    """Nodes of Algorithm 1 on P~ with the split m = l + floor((r-l)/2).

    Step 1 of Algorithm 1 ("rows of the inverse") for each node, by definition:
    block row m of the inverse of the node's sub-matrix {P~}_l^r (notation of
    Section 2.1), computed here by dense inversion.  Stored once and reused for
    every right-hand side."""
    S, M, _ = Ct.shape
    nodes: List[Node] = []
    stack = [(0, S - 1, 0)]
    while stack:
        l, r, lev = stack.pop(0)
        if l > r:
            continue
        m = l + (r - l) // 2
        P = dense_P(At[l:r + 1].copy(), Bt[l:r + 1].copy(), Ct[l:r + 1].copy())
        Pinv = np.linalg.inv(P)
        row = Pinv[(m - l) * M:(m - l + 1) * M]  # [M, n*M]
        R = np.stack([row[:, t * M:(t + 1) * M] for t in range(r - l + 1)])
        HL = R[0] @ At[l] if l > 0 else np.zeros((M, M))
        HR = R[-1] @ Bt[r] if r < S - 1 else np.zeros((M, M))
        nodes.append(Node(l, r, m, lev, R, HL, HR))
        stack.append((l, m - 1, lev + 1))
        stack.append((m + 1, r, lev + 1))
    return nodes


def dichotomy_solve(At, Ct, Bt, Ft):
    """X~ from P~ X~ = F~ by Algorithm 1: the middle unknown of a subsystem from
    the stored row of its inverse applied to its right-hand side, then the two
    subsystems with that right-hand side modified at their end blocks by
    Bt_{m-1} X~_m (left half, eq. suba) and At_{m+1} X~_m (right half, eq. subb)."""
    S, M, K = Ft.shape
    nodes = {(n.l, n.r): n for n in dichotomy_tree(At, Ct, Bt)}
    X = np.zeros((S, M, K))
    work = [(0, S - 1, Ft.copy())]
    while work:
        l, r, rhs = work.pop(0)
        if l > r:
            continue
        node = nodes[(l, r)]
        m = node.m
        X[m] = np.einsum("tab,tbk->ak", node.R, rhs[l:r + 1])
        if l <= m - 1:
            left = rhs.copy()
            left[m - 1] = left[m - 1] + Bt[m - 1] @ X[m]
            work.append((l, m - 1, left))
        if m + 1 <= r:
            right = rhs.copy()
            right[m + 1] = right[m + 1] + At[m + 1] @ X[m]
            work.append((m + 1, r, right))
    return X


def alg2_solve(A, B, C, F, S, return_parts=False):
    """Algorithm 2, stage 2: W (eq. sub3), P~ X~ = F~ by Algorithm 1 (eq. red1),
    then X_i = U_i X~_s + V_i X~_{s+1} + W_i (eq. superposition, X~_S = X_{N+1} = 0)."""
    N, M, K = F.shape
    L = N // S
    U, V = segment_responses(A, B, C, S)
    W = segment_W(A, B, C, F, S)
    At, Ct, Bt = reduced_system(A, B, C, S, U, V)
    Ft = reduced_rhs(A, B, F, W, S)
    Xt = dichotomy_solve(At, Ct, Bt, Ft)
    X = np.empty((N, M, K))
    for s, (k, a, b) in enumerate(segment_rows(N, S)):
        X[k] = Xt[s]
        right = Xt[s + 1] if s + 1 < S else np.zeros((M, K))
        for i in range(a, b):
            X[i] = U[i] @ Xt[s] + V[i] @ right + W[i]
    if return_parts:
        return X, dict(U=U, V=V, W=W, At=At, Ct=Ct, Bt=Bt, Ft=Ft, Xt=Xt)
    return X
