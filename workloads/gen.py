"""Seeded generators for the five workload shapes of the block-tridiagonal solve.

Layout (shared by every consumer):
  A, B, C : float64 [N, M, M], block j of the system
            -A_j X_{j-1} + C_j X_j - B_j X_{j+1} = F_j   (Section 2, eq. main-eq)
            A[0] and B[N-1] are unused by the system and are stored as zeros.
  F, X    : float64 [N, M, K] -- the (N*M) x K right-hand-side panel, K contiguous.

Every right-hand-side column is drawn from its own counter-seeded stream
(``default_rng([seed, column])``), so any subset of columns can be regenerated
bit-identically without drawing the rest.  Nothing here solves, factors or
applies the operator: the only arithmetic is the drawing of inputs and, for the
manufactured Poisson solutions, the textbook eigen-pairs of the five-point
Laplacian that define the inputs.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    N: int
    M: int
    K: int
    S: int
    A: np.ndarray
    B: np.ndarray
    C: np.ndarray
    F: np.ndarray
    X_exact: Optional[np.ndarray] = None  # closed-form solution, when one exists
    structure: str = "dense"  # "dense" or "stencil" (A = B = I, C tridiagonal)

    @property
    def unknowns(self) -> int:
        return self.N * self.M * self.K


@dataclasses.dataclass
class RhsSet:
    matrix: int  # index of the matrix this set is solved against
    K: int
    F: np.ndarray


# ---------------------------------------------------------------------------
# Diagonally dominant random blocks (workload "tiny random" and its larger kin)
# ---------------------------------------------------------------------------

def dominant_blocks(N: int, M: int, seed: int):
    """A_j, B_j ~ U[0,1); C_j off-diagonal ~ U[-0.5,0.5); diag(C_j) = row sums of
    |A_j|, |B_j| and |offdiag C_j| + 1 + U[0,1).  Draw order: A, B, C, diagonal
    noise.  A_1 and B_N are zeroed after drawing and excluded from the sums."""
    rng = np.random.default_rng(seed)
    A = rng.random((N, M, M))
    B = rng.random((N, M, M))
    C = rng.random((N, M, M)) - 0.5
    noise = rng.random((N, M))
    A[0] = 0.0
    B[N - 1] = 0.0
    idx = np.arange(M)
    C[:, idx, idx] = 0.0
    diag = (np.abs(A).sum(axis=2) + np.abs(B).sum(axis=2) + np.abs(C).sum(axis=2)
            + 1.0 + noise)
    C[:, idx, idx] = diag
    return A, B, C


def band_matrix(n: int, kl: int, ku: int, seed: int):
    """Diagonally dominant band matrix of order n in diagonal-ordered storage
    ab [kl + ku + 1, n], ab[ku + i - j, j] = Q[i, j]: off-diagonal entries
    ~ U[-1, 1), Q[i, i] = sum of |off-diagonal| of row i + 1 + U[0, 1).  The
    positions of ab outside the matrix are zero."""
    rng = np.random.default_rng(seed)
    ab = rng.random((kl + ku + 1, n)) * 2.0 - 1.0
    noise = rng.random(n)
    cols = np.arange(n)
    rowsum = np.zeros(n)
    for d in range(kl + ku + 1):
        rows = cols + d - ku  # row i of entry ab[d, j]
        ok = (rows >= 0) & (rows < n)
        ab[d, ~ok] = 0.0
        if d != ku:
            rowsum[rows[ok]] += np.abs(ab[d, ok])  # distinct rows within one diagonal
    ab[ku] = rowsum + 1.0 + noise
    return ab


def dominant_blocks_device(N: int, M: int, seed: int, device):
    """The distribution of `dominant_blocks`, drawn on a torch device (for the
    paper-sized shapes, whose blocks reach tens of GB): A_j, B_j ~ U[0,1),
    C_j off-diagonal ~ U[-0.5,0.5), diag(C_j) = row sums of |A_j|, |B_j| and
    |offdiag C_j| + 1 + U[0,1); A_1 and B_N zeroed.  Draw order as there, from
    one torch generator seeded with `seed` (values differ from the numpy draw)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    kw = dict(dtype=torch.float64, device=device, generator=g)
    A = torch.rand((N, M, M), **kw)
    B = torch.rand((N, M, M), **kw)
    C = torch.rand((N, M, M), **kw) - 0.5
    noise = torch.rand((N, M), **kw)
    A[0] = 0.0
    B[N - 1] = 0.0
    idx = torch.arange(M, device=device)
    C[:, idx, idx] = 0.0
    C[:, idx, idx] = A.abs().sum(dim=2) + B.abs().sum(dim=2) + C.abs().sum(dim=2) + 1.0 + noise
    return A, B, C


def uniform_rhs(N: int, M: int, K: int, seed: int,
                columns: Optional[Sequence[int]] = None, lo=-1.0, hi=1.0) -> np.ndarray:
    cols = range(K) if columns is None else columns
    F = np.empty((N, M, len(cols)))
    for c, k in enumerate(cols):
        F[:, :, c] = np.random.default_rng([seed, int(k)]).uniform(lo, hi, (N, M))
    return F


# ---------------------------------------------------------------------------
# Five-point Poisson operator with manufactured sine-mode solutions
# ---------------------------------------------------------------------------

def _tridiag_blocks(N: int, M: int, diag: np.ndarray):
    """A_j = B_j = I (dense storage), C_j = tridiag(-1, diag[j], -1)."""
    A = np.zeros((N, M, M))
    idx = np.arange(M)
    A[:, idx, idx] = 1.0
    B = A.copy()
    A[0] = 0.0
    B[N - 1] = 0.0
    C = np.zeros((N, M, M))
    C[:, idx, idx] = diag
    C[:, idx[1:], idx[:-1]] = -1.0
    C[:, idx[:-1], idx[1:]] = -1.0
    return A, B, C


def poisson_system(N: int, M: int):
    return _tridiag_blocks(N, M, np.full((N, M), 4.0))


def poisson_manufactured(N: int, M: int, K: int, seed: int, n_modes: int = 8,
                         columns: Optional[Sequence[int]] = None):
    """Per column: n_modes sine modes phi_{p,q}(i,j) = sin(p pi i/(M+1)) sin(q pi j/(N+1))
    with (p, q) uniform over [1..M] x [1..N] and amplitudes a ~ U[-1,1].
    Returns (X_exact, F) with F = sum a * lambda_{p,q} * phi_{p,q}, where
    lambda_{p,q} = 4 - 2 cos(p pi/(M+1)) - 2 cos(q pi/(N+1)) is the eigenvalue
    of the five-point operator for that mode (separation of variables)."""
    cols = range(K) if columns is None else columns
    X = np.zeros((N, M, len(cols)))
    F = np.zeros((N, M, len(cols)))
    i = np.arange(1, M + 1)
    j = np.arange(1, N + 1)
    for c, k in enumerate(cols):
        rng = np.random.default_rng([seed, int(k)])
        p = rng.integers(1, M + 1, n_modes)
        q = rng.integers(1, N + 1, n_modes)
        a = rng.uniform(-1.0, 1.0, n_modes)
        for t in range(n_modes):
            si = np.sin(p[t] * math.pi * i / (M + 1))
            sj = np.sin(q[t] * math.pi * j / (N + 1))
            lam = 4.0 - 2.0 * math.cos(p[t] * math.pi / (M + 1)) - 2.0 * math.cos(q[t] * math.pi / (N + 1))
            mode = np.outer(sj, si)  # [N, M]
            X[:, :, c] += a[t] * mode
            F[:, :, c] += a[t] * lam * mode
    return X, F


# ---------------------------------------------------------------------------
# Acoustic-style shifted operator with a quadratic absorbing-layer profile
# ---------------------------------------------------------------------------

def pml_sigma(n: int, width: int = 20, peak: float = 2.0) -> np.ndarray:
    """Quadratic (nu = 2) damping profile over the last `width` points at each
    edge of an n-point line, rising from ~0 to `peak` at the outermost point.
    Point k (1-based): t = (width+1-k)/width for k <= width,
    t = (k-(n-width))/width for k > n-width, 0 otherwise; sigma = peak * t^2."""
    k = np.arange(1, n + 1, dtype=np.float64)
    t = np.zeros(n)
    lo = k <= width
    hi = k > n - width
    t[lo] = (width + 1 - k[lo]) / width
    t[hi] = (k[hi] - (n - width)) / width
    return peak * t * t


def acoustic_system(N: int, M: int, shift: float = 0.25):
    sig = pml_sigma(N)[:, None] + pml_sigma(M)[None, :]
    return _tridiag_blocks(N, M, 4.0 + shift + sig)


def source_wavelet(t: np.ndarray, f0=30.0, t0=0.2, g=4.0) -> np.ndarray:
    """Source time function of the paper's acoustic experiment (eq. functiont)."""
    arg = 2.0 * math.pi * f0 * (t - t0)
    return np.exp(-(arg * arg) / (g * g)) * np.sin(arg)


def acoustic_rhs(N: int, M: int, K: int, seed: int, n_src: int = 16,
                 noise: float = 1e-3, columns: Optional[Sequence[int]] = None) -> np.ndarray:
    """Column m: n_src random grid points get f(t_m) * u, u ~ U[0.5, 1],
    t_m = 0.4 m / (K-1) s, plus noise * N(0,1) everywhere."""
    cols = range(K) if columns is None else columns
    F = np.empty((N, M, len(cols)))
    for c, k in enumerate(cols):
        rng = np.random.default_rng([seed, int(k)])
        col = noise * rng.standard_normal((N, M))
        jj = rng.integers(0, N, n_src)
        ii = rng.integers(0, M, n_src)
        u = rng.uniform(0.5, 1.0, n_src)
        tm = 0.4 * k / max(K - 1, 1)
        amp = float(source_wavelet(np.array([tm]))[0])
        np.add.at(col, (jj, ii), amp * u)
        F[:, :, c] = col
    return F


# ---------------------------------------------------------------------------
# Uneven right-hand-side sets against several matrices
# ---------------------------------------------------------------------------

def batched_K(n_sets: int, seed: int, kmax: int = 1024) -> List[int]:
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, math.log(kmax), n_sets)
    return [int(min(max(round(math.exp(x)), 1), kmax)) for x in u]


def batched_sets(N: int, M: int, n_mats: int = 4, n_sets: int = 64, seed: int = 5,
                 kmax: int = 1024, mat_seeds: Optional[Sequence[int]] = None):
    """n_mats diagonally dominant matrices (seeds 1..n_mats by default) and
    n_sets right-hand-side sets with K log-uniform on [1, kmax]; set b uses
    matrix b mod n_mats.  Returns (mats, sets)."""
    mat_seeds = list(mat_seeds) if mat_seeds is not None else list(range(1, n_mats + 1))
    mats = [dominant_blocks(N, M, s) for s in mat_seeds]
    Ks = batched_K(n_sets, seed, kmax)
    sets = [RhsSet(matrix=b % n_mats, K=Ks[b], F=uniform_rhs(N, M, Ks[b], seed=1000 * seed + b))
            for b in range(n_sets)]
    return mats, sets


# ---------------------------------------------------------------------------
# The five named workloads
# ---------------------------------------------------------------------------

def config0(seed: int = 0) -> Workload:
    """Tiny random system: N=64, M=4, K=1, S=8."""
    N, M, K, S = 64, 4, 1, 8
    A, B, C = dominant_blocks(N, M, seed)
    F = uniform_rhs(N, M, K, seed=seed + 100)
    return Workload("tiny-random N64 M4 K1 S8", N, M, K, S, A, B, C, F)


def config1(N: int = 1024, M: int = 256, K: int = 64, S: int = 64, seed: int = 1,
            columns: Optional[Sequence[int]] = None) -> Workload:
    """Five-point Poisson operator, manufactured sine-mode solutions."""
    A, B, C = poisson_system(N, M)
    X, F = poisson_manufactured(N, M, K, seed, columns=columns)
    return Workload(f"poisson N{N} M{M} K{K} S{S}", N, M, F.shape[2], S, A, B, C, F,
                    X_exact=X, structure="stencil")


def config2(N: int = 4096, M: int = 128, K: int = 512, S: int = 64, seed: int = 2,
            columns: Optional[Sequence[int]] = None) -> Workload:
    """Shifted acoustic-style operator with absorbing-layer damping, 512 harmonics."""
    A, B, C = acoustic_system(N, M)
    F = acoustic_rhs(N, M, K, seed, columns=columns)
    return Workload(f"acoustic N{N} M{M} K{K} S{S}", N, M, F.shape[2], S, A, B, C, F,
                    structure="stencil")


def config3(N: int = 2048, M: int = 64, n_sets: int = 64, n_mats: int = 4, kmax: int = 1024):
    """Four diagonally dominant matrices, 64 uneven right-hand-side sets."""
    return batched_sets(N, M, n_mats=n_mats, n_sets=n_sets, kmax=kmax)


def config4(N: int = 2048, M: int = 64, K: int = 128, seed: int = 4):
    """Matrix, right-hand sides and regression target of the gradient workload."""
    A, B, C = dominant_blocks(N, M, seed)
    F = uniform_rhs(N, M, K, seed=seed + 100)
    Xt = uniform_rhs(N, M, K, seed=seed + 200)
    return A, B, C, F, Xt
