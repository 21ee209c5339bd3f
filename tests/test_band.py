"""Band matrices through the block-tridiagonal solver (GPU only).

Section 3.3.1, item c: the PML operator is a band matrix that the dichotomy
solves as a block-tridiagonal system with triangular off-diagonal blocks.
bt_factor_band cuts a band matrix (diagonal-ordered storage) into M x M
blocks on the device; every factorisation detects the diagonal bands of its
A_j and B_j and contracts its GEMMs over them only.  Checked against the
oracle's block form (block Thomas) and LAPACK's banded LU, element by element.
"""

import ctypes

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import band as oband
from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def bt():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1108_4181_gb300 as bt

    return bt


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _band_of(X, first, last):
    """(lo, hi) of c - r over the nonzero entries of blocks first..last; (0, 0) if none."""
    M = X.shape[1]
    d = np.arange(M)[None, :] - np.arange(M)[:, None]
    nz = (X[first:last + 1] != 0).any(axis=0)
    return (int(d[nz].min()), int(d[nz].max())) if nz.any() else (0, 0)


# (n, kl, ku, M, S, K): full band with n = N M; ragged n; the PML shape (band
# 3 x 30, M = 128); tridiagonal; no sub-diagonals (A_j = 0); M = 150 (32-wide
# GEMM tiles)
CASES = [(2048, 64, 64, 64, 8, 3), (1000, 7, 3, 64, 4, 5), (3600, 90, 90, 128, 4, 2), (257, 1, 1, 8, 8, 1),
         (500, 0, 2, 16, 2, 2), (700, 150, 150, 150, 2, 2)]


@pytest.mark.parametrize("n,kl,ku,M,S,K", CASES)
def test_band_parity(bt, n, kl, ku, M, S, K):
    ab = gen.band_matrix(n, kl, ku, seed=n + kl)
    F = np.random.default_rng(n).uniform(-1, 1, (n, K))
    A, B, C, N = oband.band_blocks(ab, kl, ku, M, S)
    Xr = oracle.solve_block_thomas(A, B, C, oband.pad_rows(F, N, M)).reshape(N * M, K)[:n]
    Xl = scipy.linalg.solve_banded((kl, ku), ab, F)
    ab_dev = ab.copy()
    for d in range(kl + ku + 1):  # positions outside the matrix are never read
        cols = np.arange(n)
        ab_dev[d, (cols + d - ku < 0) | (cols + d - ku >= n)] = np.nan
    with bt.factor_band(_t(ab_dev), kl, ku, M, S) as fac:
        assert (fac.N, fac.M, fac.n) == (N, M, n)
        info = fac.band()
        X = fac.solve(_t(F)).cpu().numpy()
    assert info["A"] == _band_of(A, 1, N - 1) and info["B"] == _band_of(B, 0, N - 2)
    assert info["A"][0] >= M - kl or kl == 0  # upper triangular A_j
    assert info["B"][1] <= ku - M or ku == 0  # lower triangular B_j
    assert oracle.rel_err(X, Xr) <= 1e-12
    assert oracle.col_err(X, Xr) <= 1e-12
    assert oracle.rel_err(X, Xl) <= 1e-12
    assert oracle.col_err(X, Xl) <= 1e-12


@pytest.mark.parametrize("n", [2560, 2500])
def test_band_refined(bt, n):
    # split-BF16 refinement with the tensor-core residual on a band matrix of
    # half-bandwidth 64 (M = 64), n a multiple of M and ragged
    kl = ku = 64
    ab = gen.band_matrix(n, kl, ku, seed=3)
    F = np.random.default_rng(7).uniform(-1, 1, (n, 150))
    A, B, C, N = oband.band_blocks(ab, kl, ku, 64, 8)
    Xr = oracle.solve_block_thomas(A, B, C, oband.pad_rows(F, N, 64)).reshape(N * 64, -1)[:n]
    with bt.factor_band(_t(ab), kl, ku, 64, 8) as fac:
        X, info = fac.solve(_t(F), precision="bf16x3", tol=1e-11, return_info=True)
    assert info["converged"]
    assert oracle.rel_err(X.cpu().numpy(), Xr) <= 1e-10
    assert oracle.col_err(X.cpu().numpy(), Xr) <= 1e-10


def test_band_vector_rhs_and_out(bt):
    n, kl, ku = 300, 4, 9
    ab = gen.band_matrix(n, kl, ku, seed=1)
    f = np.random.default_rng(2).uniform(-1, 1, n)
    with bt.factor_band(_t(ab), kl, ku, 16, 4) as fac:
        x = fac.solve(_t(f))
        out = torch.empty(n, dtype=torch.float64, device=DEV)
        x2 = fac.solve(_t(f), out=out)
    assert x.shape == (n,) and x2.data_ptr() == out.data_ptr()
    xl = scipy.linalg.solve_banded((kl, ku), ab, f)
    assert oracle.rel_err(x.cpu().numpy(), xl) <= 1e-12
    assert oracle.col_err(x.cpu().numpy(), xl) <= 1e-12
    assert torch.equal(x, out)


@pytest.mark.parametrize("M", [40, 128, 150])
def test_band_detection_general_blocks(bt, M):
    # bt_factor on blocks whose A_j / B_j are zero outside diagonal bands that
    # do not start at the main diagonal: the detected bands are exact and the
    # shortened GEMM contractions give the oracle's solution
    N, S, K = 16, 4, 3
    rng = np.random.default_rng(M)
    d = np.arange(M)[None, :] - np.arange(M)[:, None]
    A = rng.uniform(0.1, 1.0, (N, M, M)) * ((d >= 5) & (d <= 20))
    B = rng.uniform(0.1, 1.0, (N, M, M)) * ((d >= -30) & (d <= -3))
    C = rng.uniform(-0.5, 0.5, (N, M, M))
    A[0] = 0.0
    B[N - 1] = 0.0
    idx = np.arange(M)
    C[:, idx, idx] = np.abs(A).sum(2) + np.abs(B).sum(2) + np.abs(C).sum(2) + 1.0
    F = gen.uniform_rhs(N, M, K, seed=M)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        info = fac.band()
        X = fac.solve(_t(F)).cpu().numpy()
    assert info["A"] == (5, 20) and info["B"] == (-30, -3) and info["n"] == 0
    assert oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-12
    assert oracle.col_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-12


def test_band_detection_dense_and_stencil(bt):
    A, B, C = gen.dominant_blocks(8, 24, seed=2)
    with bt.factor(_t(A), _t(B), _t(C), 2) as fac:
        assert fac.band()["A"] == (-23, 23) and fac.band()["B"] == (-23, 23)
    A, B, C = gen.poisson_system(8, 24)
    with bt.factor(_t(A), _t(B), _t(C), 2) as fac:
        assert fac.band()["A"] == (0, 0) and fac.band()["B"] == (0, 0)


def test_band_rejects_bad_arguments(bt):
    lib = bt._lib.load()
    ab = _t(gen.band_matrix(100, 3, 3, seed=1))
    h = ctypes.c_void_p()
    name = lambda st: bt._lib.STATUS_NAMES.get(st)  # noqa: E731
    P = bt.solver._ptr
    assert name(lib.bt_factor_band(100, 9, 3, P(ab), 8, 1, None, ctypes.byref(h))) == "BT_ERR_ARG"  # kl > M
    assert name(lib.bt_factor_band(100, 3, 3, P(ab), 8, 14, None, ctypes.byref(h))) == "BT_ERR_ARG"  # S > 13
    assert name(lib.bt_factor_band(0, 3, 3, P(ab), 8, 1, None, ctypes.byref(h))) == "BT_ERR_ARG"
    assert name(lib.bt_factor_band(100, 3, 3, None, 8, 1, None, ctypes.byref(h))) == "BT_ERR_ARG"
    F = _t(np.ones((100, 2)))
    with bt.factor_band(ab, 3, 3, 8, 2) as fac:
        st = lib.bt_solve_band(fac._h, P(F), 2, P(F), None, None)  # X overlapping F
        assert name(st) == "BT_ERR_ARG"
    A, B, C = gen.dominant_blocks(4, 8, seed=1)
    with bt.factor(_t(A), _t(B), _t(C), 2) as fac:  # not a band handle
        X = torch.empty_like(F)
        assert name(lib.bt_solve_band(fac._h, P(F), 2, P(X), None, None)) == "BT_ERR_ARG"
