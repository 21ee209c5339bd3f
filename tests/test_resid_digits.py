"""The exact tensor-core residual (bt_residual method "digits") vs the CPU oracle (GPU only).

r = F - P X is formed from seven balanced base-128 digits of every operator
row and every column of X (one power-of-two scale each), exact FP32 digit
products on the tensor cores and 64-bit integer combination.  Its error bound
per entry is 7.5 M 2^(e_A + e_X - 49), where 2^e_A exceeds the largest |entry|
of row m of A_j, B_j, C_j and 2^e_X the largest |X| of the column; the tests
recompute both scales from that definition and hold every entry to the bound
(the oracle's own FP64 rounding is far below it).  An inexact accumulation in
any of the four leading digit sums would exceed the bound by orders of
magnitude.
"""

import numpy as np
import pytest

import oracle
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


def _scale(mx):
    """e with |v| < 2^e for a set whose largest magnitude is mx (0 for zero)."""
    _, e = np.frexp(mx)
    return np.where(mx > 0, e, 0)


def _bound(A, B, C, X):
    """Per-entry bound 7.5 M 2^(e_A(j,m) + e_X(n) - 49), shape [N, M, K]."""
    M = C.shape[1]
    ea = _scale(np.maximum(np.maximum(np.abs(A).max(axis=2), np.abs(B).max(axis=2)), np.abs(C).max(axis=2)))
    ex = _scale(np.abs(X).max(axis=(0, 1)))
    return 7.5 * M * np.ldexp(1.0, ea[:, :, None] + ex[None, None, :] - 49)


def _check(A, B, C, X, F, R, n2):
    Rr = oracle.residual(A, B, C, X, F)
    err = np.abs(R - Rr)
    bound = _bound(A, B, C, X)
    worst = float((err / bound).max())
    assert worst <= 1.0, worst
    assert abs(n2 - float((Rr ** 2).sum())) <= 1e-6 * float((Rr ** 2).sum()) + 1e-300
    return worst


@pytest.mark.parametrize("M", [64, 128])
@pytest.mark.parametrize("K", [1, 37, 300])
def test_digits_random_x(bt, M, K):
    # X unrelated to F: r of the size of F, no cancellation
    N = 7
    A, B, C = gen.dominant_blocks(N, M, seed=M + K)
    F = gen.uniform_rhs(N, M, K, seed=3)
    X = gen.uniform_rhs(N, M, K, seed=4)
    with bt.factor(_t(A), _t(B), _t(C), 1) as fac:
        R, n2 = fac.residual(_t(F), _t(X), method="digits")
    _check(A, B, C, X, F, R.cpu().numpy(), n2)


@pytest.mark.parametrize("M", [64, 128])
def test_digits_near_solution(bt, M):
    # X = solution + 1e-6 relative perturbation: r about 1e-6 |F|, the
    # cancellation the refinement meets; also against the FP64 CUDA-core path
    N, K = 9, 130
    A, B, C = gen.dominant_blocks(N, M, seed=M)
    F = gen.uniform_rhs(N, M, K, seed=5)
    X = oracle.solve_block_thomas(A, B, C, F)
    X = X * (1.0 + 1e-6 * np.random.default_rng(1).standard_normal(X.shape))
    with bt.factor(_t(A), _t(B), _t(C), 3) as fac:
        R, n2 = fac.residual(_t(F), _t(X), method="digits")
        R64, n64 = fac.residual(_t(F), _t(X), method="fp64")
    Rr = oracle.residual(A, B, C, X, F)
    _check(A, B, C, X, F, R.cpu().numpy(), n2)
    assert np.abs(R64.cpu().numpy() - Rr).max() <= 1e-13 * np.abs(F).max()


def test_digits_large_sums_wrap(bt):
    # every entry positive and near its row / column maximum: the digit sums
    # approach their bound (3M * 2^14 for the leading digits) and the product
    # term exceeds 2^63 units, so the 64-bit combination wraps; F = P X + small
    # keeps r representable, and r must still be exact within the bound
    N, M, K = 5, 128, 64
    rng = np.random.default_rng(7)
    A = rng.uniform(0.75, 1.0, (N, M, M))
    B = rng.uniform(0.75, 1.0, (N, M, M))
    C = -rng.uniform(0.75, 1.0, (N, M, M))
    A[0] = 0.0
    B[N - 1] = 0.0
    X = rng.uniform(0.75, 1.0, (N, M, K))
    F = oracle.apply_P(A, B, C, X) + rng.uniform(-1e-3, 1e-3, (N, M, K))
    with bt.factor(_t(A), _t(B), _t(C), 1) as fac:
        R, n2 = fac.residual(_t(F), _t(X), method="digits")
    _check(A, B, C, X, F, R.cpu().numpy(), n2)


def test_digits_scales_and_special_columns(bt):
    # rows of very different magnitude, a zero column of X (r = F there), a
    # column of X with a huge scale, and F far larger than P X in one column
    N, M, K = 6, 64, 5
    A, B, C = gen.dominant_blocks(N, M, seed=9)
    row_scale = np.ldexp(1.0, np.random.default_rng(2).integers(-30, 30, (N, M)))
    A, B, C = (a * row_scale[:, :, None] for a in (A, B, C))
    X = gen.uniform_rhs(N, M, K, seed=6)
    X[:, :, 1] = 0.0
    X[:, :, 2] *= 1e200
    F = gen.uniform_rhs(N, M, K, seed=8)
    F[:, :, 3] *= 1e40
    with bt.factor(_t(A), _t(B), _t(C), 2) as fac:
        R, n2 = fac.residual(_t(F), _t(X), method="digits")
    R = R.cpu().numpy()
    Rr = oracle.residual(A, B, C, X, F)  # column 1: r = F
    bound = _bound(A, B, C, X) + 1e-15 * np.abs(Rr)
    assert (np.abs(R - Rr) <= bound).all()


def test_digits_nan_column(bt):
    # a non-finite X column poisons its own residual column and the norm only
    N, M, K = 4, 64, 3
    A, B, C = gen.dominant_blocks(N, M, seed=1)
    F = gen.uniform_rhs(N, M, K, seed=2)
    X = gen.uniform_rhs(N, M, K, seed=3)
    X[2, 5, 1] = np.nan
    with bt.factor(_t(A), _t(B), _t(C), 1) as fac:
        R, n2 = fac.residual(_t(F), _t(X), method="digits")
    R = R.cpu().numpy()
    assert np.isnan(R[:, :, 1]).all()
    assert np.isnan(n2)
    Rr = oracle.residual(A, B, C, X[:, :, [0, 2]], F[:, :, [0, 2]])
    assert np.abs(R[:, :, [0, 2]] - Rr).max() <= _bound(A, B, C, X[:, :, [0, 2]]).max()


def test_digits_unsupported(bt):
    N, M = 8, 16
    A, B, C = gen.dominant_blocks(N, M, seed=1)
    F = gen.uniform_rhs(N, M, 2, seed=2)
    with bt.factor(_t(A), _t(B), _t(C), 2) as fac:
        with pytest.raises(bt.BtError) as e:
            fac.residual(_t(F), _t(F), method="digits")
        assert e.value.name == "BT_ERR_UNSUPPORTED"
        R, _ = fac.residual(_t(F), _t(F), method="auto")  # falls back to FP64
    Rr = oracle.residual(A, B, C, F, F)
    assert np.abs(R.cpu().numpy() - Rr).max() <= 1e-13 * np.abs(Rr).max()


def test_digits_full_size_sampled(bt):
    # the uneven-set workload's matrix size (N = 2048, M = 64) at K = 300, in
    # the launch configuration of the refined solve; sampled columns
    N, M, K = 2048, 64, 300
    A, B, C = gen.dominant_blocks(N, M, seed=1)
    F = gen.uniform_rhs(N, M, K, seed=11)
    cols = [0, 1, 127, 128, 255, 299]
    with bt.factor(_t(A), _t(B), _t(C), 32) as fac:
        Xd = fac.solve(_t(F))
        Xd = Xd * (1.0 + 1e-7 * torch.randn_like(Xd))
        R, n2 = fac.residual(_t(F), Xd, method="digits")
    X = Xd[:, :, cols].cpu().numpy()
    Rr = oracle.residual(A, B, C, X, F[:, :, cols])
    # e_X depends on the column alone: the bound of the sampled columns
    assert (np.abs(R[:, :, cols].cpu().numpy() - Rr) <= _bound(A, B, C, X)).all()


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32", "f32"])
def test_refined_solve_with_digit_residual(bt, prec):
    # the refinement on dense blocks with the exact tensor-core residual: the
    # device's reported residual agrees with the oracle's, and the solution
    # matches the FP64 oracle
    N, M, K, S = 64, 64, 150, 8
    A, B, C = gen.dominant_blocks(N, M, seed=21)
    F = gen.uniform_rhs(N, M, K, seed=22)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        X, info = fac.solve(_t(F), precision=prec, tol=1e-11, residual="digits", return_info=True)
        X2, info2 = fac.solve(_t(F), precision=prec, tol=1e-11, residual="fp64", return_info=True)
    X = X.cpu().numpy()
    assert info["converged"] and info2["converged"]
    rr = oracle.rel_res(A, B, C, X, F)
    assert rr <= 2e-11
    # agreement to 0.1 %, down to the FP64 noise floor of these systems (the
    # solve overshoots the tolerance to ~1e-14, where both residuals are
    # rounding-limited)
    assert abs(info["rel_res"] - rr) <= 1e-3 * rr + 1e-13
    Xr = oracle.solve_block_thomas(A, B, C, F)
    assert oracle.rel_err(X, Xr) <= 1e-10
    assert oracle.col_err(X, Xr) <= 1e-10
    assert oracle.rel_err(X2.cpu().numpy(), Xr) <= 1e-10
    assert oracle.col_err(X2.cpu().numpy(), Xr) <= 1e-10


def test_residual_rejects_bad_arguments(bt):
    N, M = 8, 64
    A, B, C = gen.dominant_blocks(N, M, seed=1)
    F = _t(gen.uniform_rhs(N, M, 2, seed=2))
    with bt.factor(_t(A), _t(B), _t(C), 2) as fac:
        lib = bt._lib.load()
        R = torch.empty_like(F)
        for args in [(F, F, F), (F, R, R)]:  # R aliasing F or X
            st = lib.bt_residual(fac._h, bt.solver._ptr(args[0]), bt.solver._ptr(args[1]), 2,
                                 bt.solver._ptr(args[2]), 2, None, None)
            assert bt._lib.STATUS_NAMES.get(st) == "BT_ERR_ARG"
        st = lib.bt_residual(fac._h, bt.solver._ptr(F), bt.solver._ptr(F), 2, bt.solver._ptr(R), 5, None, None)
        assert bt._lib.STATUS_NAMES.get(st) == "BT_ERR_ARG"  # unknown method
