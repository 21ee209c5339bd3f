"""Schur-complement CG with a probing band preconditioner, in FP64 on the CPU
(test infrastructure).

Section 3.3 (Domain decomposition): the interface unknowns x_G of a
non-overlapping decomposition solve the Schur-complement system of eq.
schur_decomp, S x_G = f_G - sum_i A_Gi A_ii^{-1} f_i with
S = A_GG - sum_i A_Gi A_ii^{-1} A_iG, by the conjugate gradient method without
forming S (each product with S inverts every A_ii); the interiors follow from
eq. domains_equation, x_i = A_ii^{-1} (f_i - A_iG x_G).  Section 3.3.2
preconditions the CG by a band matrix B of half-bandwidth d built by probing:
B is read off the products S p_l with the 2d+1 vectors p_l that are 1 on the
indices congruent to l modulo 2d+1, and B is inverted by the dichotomy.

The model problem (a stand-in for the paper's layered medium): the five-point
operator (4 + shift) x_{z,r} - x_{z-1,r} - x_{z+1,r} - x_{z,r-1} - x_{z,r+1}
on an nz x nr grid with zero Dirichlet values outside, cut by p - 1 grid rows
(the interface lines) into p strips of h rows: nz = p h + p - 1, strip i holds
rows i (h + 1) .. i (h + 1) + h - 1, interface line k is row k (h + 1) + h.
Panels are [nz, nr, K] (grid row-major, K right-hand sides); interface panels
[p - 1, nr, K].  Each strip operator, with its unknowns ordered by grid column
(block j = column r, M = h), is block tridiagonal with A_j = B_j = I and
C_j = tridiag(-1, 4 + shift, -1): the form the dichotomy solves.
"""

from __future__ import annotations

import numpy as np

from .blocktri import solve_block_thomas


def grid_rows(h: int, p: int):
    """(nz, strip row lists, interface rows) of the cut."""
    nz = p * h + p - 1
    strips = [list(range(i * (h + 1), i * (h + 1) + h)) for i in range(p)]
    iface = [k * (h + 1) + h for k in range(p - 1)]
    return nz, strips, iface


def _tridiag(n: int, diag: float):
    T = np.diag(np.full(n, diag))
    if n > 1:
        T += np.diag(np.full(n - 1, -1.0), 1) + np.diag(np.full(n - 1, -1.0), -1)
    return T


def grid_blocks(nr: int, nz: int, shift: float):
    """The whole grid operator as a block-tridiagonal system over grid rows
    (block j = row z, M = nr): A_j = B_j = I, C_j = tridiag(-1, 4 + shift, -1)."""
    A = np.broadcast_to(np.eye(nr), (nz, nr, nr)).copy()
    B = A.copy()
    A[0] = 0.0
    B[nz - 1] = 0.0
    C = np.broadcast_to(_tridiag(nr, 4.0 + shift), (nz, nr, nr)).copy()
    return A, B, C


def strip_blocks(nr: int, h: int, shift: float):
    """A strip operator over grid columns (block j = column r, M = h)."""
    A = np.broadcast_to(np.eye(h), (nr, h, h)).copy()
    B = A.copy()
    A[0] = 0.0
    B[nr - 1] = 0.0
    C = np.broadcast_to(_tridiag(h, 4.0 + shift), (nr, h, h)).copy()
    return A, B, C


def _strip_solve(nr, h, shift, R):
    """A_ii^{-1} R for one strip; R is [h, nr, K] in grid order."""
    A, B, C = strip_blocks(nr, h, shift)
    Y = solve_block_thomas(A, B, C, np.ascontiguousarray(R.transpose(1, 0, 2)))
    return Y.transpose(1, 0, 2)


def schur_apply(v, nr: int, h: int, p: int, shift: float):
    """S v for an interface panel v [p - 1, nr, K]: A_GG v - sum_i A_Gi A_ii^{-1} A_iG v.

    A_iG v is -v on the strip rows next to each interface line; A_Gi w is -w
    read on those rows; A_GG is the five-point operator along the line."""
    K = v.shape[2]
    out = (4.0 + shift) * v
    out[:, 1:] -= v[:, :-1]
    out[:, :-1] -= v[:, 1:]
    for i in range(p):
        R = np.zeros((h, nr, K))
        if i > 0:
            R[0] -= v[i - 1]  # A_iG v: line i-1 lies above strip i
        if i < p - 1:
            R[h - 1] -= v[i]  # line i lies below strip i
        W = _strip_solve(nr, h, shift, R)
        if i > 0:
            out[i - 1] -= -W[0]  # - A_Gi W, A_Gi = -1 on the neighbouring rows
        if i < p - 1:
            out[i] -= -W[h - 1]
    return out


def schur_rhs(F, nr: int, h: int, p: int, shift: float):
    """g = f_G - sum_i A_Gi A_ii^{-1} f_i for a grid panel F [nz, nr, K]."""
    nz, strips, iface = grid_rows(h, p)
    g = F[iface].copy()
    for i in range(p):
        W = _strip_solve(nr, h, shift, F[strips[i]])
        if i > 0:
            g[i - 1] += W[0]
        if i < p - 1:
            g[i] += W[h - 1]
    return g


def recover(F, xG, nr: int, h: int, p: int, shift: float):
    """The whole grid panel from x_G (eq. domains_equation): x_i = A_ii^{-1}(f_i - A_iG x_G)."""
    nz, strips, iface = grid_rows(h, p)
    X = np.zeros_like(F)
    X[iface] = xG
    for i in range(p):
        R = F[strips[i]].copy()
        if i > 0:
            R[0] += xG[i - 1]
        if i < p - 1:
            R[h - 1] += xG[i]
        X[strips[i]] = _strip_solve(nr, h, shift, R)
    return X


def probing_vectors(n: int, d: int):
    """The 2d+1 probing vectors as columns: P[i, l] = 1 where i mod (2d+1) = l."""
    w = 2 * d + 1
    P = np.zeros((n, w))
    P[np.arange(n), np.arange(n) % w] = 1.0
    return P


def probe_band(SP, d: int):
    """Band storage ab [2d+1, n] (ab[d + i - j, j] = B[i, j]) of the probed matrix.

    B[i, j] = (S p_{j mod w})[i] for |i - j| <= d reads entry (i, j) of a
    matrix whose band is at most d (no two columns of one residue class lie
    within d of a row); S is symmetric, so the probed B is symmetrised,
    B <- (B + B^T) / 2, to keep the preconditioner symmetric for CG."""
    n = SP.shape[0]
    w = 2 * d + 1
    ab = np.zeros((w, n))
    for j in range(n):
        for i in range(max(0, j - d), min(n, j + d + 1)):
            ab[d + i - j, j] = 0.5 * (SP[i, j % w] + SP[j, i % w])
    return ab


def pcg(apply_S, solve_B, g, tol: float, max_it: int):
    """Preconditioned conjugate gradients (Saad, Algorithm 9.1) for each column
    of g [n, K] from x = 0; a column stops once ||r|| <= tol ||g||.
    Returns (x, iterations, relative residual per column)."""
    n, K = g.shape
    x = np.zeros_like(g)
    r = g.copy()
    z = solve_B(r)
    pdir = z.copy()
    rz = (r * z).sum(axis=0)
    gn = np.sqrt((g * g).sum(axis=0))
    active = np.sqrt((r * r).sum(axis=0)) > tol * gn
    it = 0
    while active.any() and it < max_it:
        q = apply_S(pdir)
        alpha = np.where(active, rz / np.where(active, (pdir * q).sum(axis=0), 1.0), 0.0)
        x += alpha * pdir
        r -= alpha * q
        it += 1
        active &= np.sqrt((r * r).sum(axis=0)) > tol * gn
        z = solve_B(r)
        rz_new = (r * z).sum(axis=0)
        beta = np.where(active, rz_new / np.where(active, rz, 1.0), 0.0)
        pdir = z + beta * pdir
        rz = rz_new
    return x, it, np.sqrt((r * r).sum(axis=0)) / np.where(gn > 0, gn, 1.0)


def grid_apply(X, shift: float):
    """A X for the five-point grid operator on a panel X [nz, nr, K] (zero outside the grid)."""
    Y = (4.0 + shift) * X
    Y[1:] -= X[:-1]
    Y[:-1] -= X[1:]
    Y[:, 1:] -= X[:, :-1]
    Y[:, :-1] -= X[:, 1:]
    return Y
