"""The FP32 double-word residual of unit-stencil operators on the GPU
(bt_residual method 3, and the refinement that uses it), entry by entry against
the oracle's FP64 residual F - P X.

Bar (the bound stated in bt.h and pinned by tests/test_dw_model.py): every
entry within 2^-23 |r| + 2^-42 S of the exact residual, S = |f| + |P||x| over
the entry's six terms; the oracle's own FP64 rounding (a few 2^-53 S) is added
as an allowance.  Out-of-range values must fall back to the FP64 residual
exactly; unsupported operators are refused.
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


def _S(F, X, C):
    """|f| + |P||x| per entry for A = B = I, tridiagonal C."""
    cd = np.abs(np.einsum("jmm->jm", C))[:, :, None]
    S = np.abs(F) + cd * np.abs(X)
    S[1:] += np.abs(X[:-1])
    S[:-1] += np.abs(X[1:])
    S[:, 1:] += np.abs(X[:, :-1])
    S[:, :-1] += np.abs(X[:, 1:])
    return S


def _check_entrywise(A, B, C, F, X, R):
    r = oracle.residual(A, B, C, X, F)
    S = _S(F, X, C)
    bound = 2.0 ** -23 * np.abs(r) + 2.0 ** -42 * S + 8 * 2.0 ** -53 * S
    err = np.abs(R - r)
    worst = float(np.max(err / bound))
    assert np.all(err <= bound), worst
    return float(np.max(err / np.maximum(S, 1e-300)))


@pytest.mark.parametrize("N,M,K,seed,what", [
    (256, 128, 40, 1, "near"),     # the acoustic operator near its solution
    (256, 128, 40, 2, "random"),
    (70, 128, 70, 3, "near"),      # N not a multiple of the 32-row march, ragged 32-column group
    (33, 8, 1, 4, "random"),       # M = 8: one row group, single column
    (40, 16, 33, 5, "near"),
])
def test_dw_residual_acoustic_entrywise(bt, N, M, K, seed, what):
    A, B, C = gen.acoustic_system(N, M)
    F = gen.acoustic_rhs(N, M, K, seed=seed)
    if what == "near":
        X = oracle.solve_block_thomas(A, B, C, F)
        X = X * (1.0 + 1e-9 * np.random.default_rng(seed).standard_normal(X.shape))
    else:
        X = np.random.default_rng(seed).uniform(-1, 1, F.shape)
    with bt.factor(_t(A), _t(B), _t(C), 1) as fac:
        R, n2 = fac.residual(_t(F), _t(X), method="dw")
        R = R.cpu().numpy()
    rel = _check_entrywise(A, B, C, F, X, R)
    if what == "near":  # r tiny against its terms: the error is the method's, not the FP32 rounding of r
        assert rel < 2.0 ** -40
    assert abs(n2 - float(np.sum(R * R))) <= 1e-5 * float(np.sum(R * R)) + 1e-300


def test_dw_residual_poisson_and_wide_magnitudes(bt):
    N, M, K = 64, 256, 5
    A, B, C = gen.poisson_system(N, M)
    rng = np.random.default_rng(9)
    X = rng.standard_normal((N, M, K)) * np.exp2(rng.integers(-60, 60, (N, M, K)))
    F = rng.standard_normal((N, M, K)) * np.exp2(rng.integers(-60, 60, (N, M, K)))
    with bt.factor(_t(A), _t(B), _t(C), 8) as fac:
        R, _ = fac.residual(_t(F), _t(X), method="dw")
    _check_entrywise(A, B, C, F, X, R.cpu().numpy())


def test_dw_residual_counts_tiny_values_as_zero(bt):
    N, M, K = 32, 16, 4
    A, B, C = gen.acoustic_system(N, M)
    rng = np.random.default_rng(10)
    X = rng.uniform(-1, 1, (N, M, K))
    X[3, 5, :] = 3e-31  # below 2^-100
    F = rng.uniform(-1, 1, (N, M, K))
    with bt.factor(_t(A), _t(B), _t(C), 4) as fac:
        R, _ = fac.residual(_t(F), _t(X), method="dw")
    R = R.cpu().numpy()
    r = oracle.residual(A, B, C, X, F)
    S = _S(F, X, C)
    assert np.all(np.abs(R - r) <= 2.0 ** -23 * np.abs(r) + 2.0 ** -42 * S + 6 * 2.0 ** -100)


def test_dw_residual_out_of_range_falls_back_to_fp64(bt):
    N, M, K = 48, 32, 6
    A, B, C = gen.acoustic_system(N, M)
    rng = np.random.default_rng(11)
    X = rng.uniform(-1, 1, (N, M, K))
    F = rng.uniform(-1, 1, (N, M, K))
    X[20, 7, 2] = 2.0 ** 80
    with bt.factor(_t(A), _t(B), _t(C), 4) as fac:
        R3, n3 = fac.residual(_t(F), _t(X), method="dw")
        R1, n1 = fac.residual(_t(F), _t(X), method="fp64")
    assert torch.equal(R3, R1) and n3 == n1
    # and a non-finite value reaches the result as in FP64
    X[1, 1, 1] = np.nan
    with bt.factor(_t(A), _t(B), _t(C), 4) as fac:
        R3, _ = fac.residual(_t(F), _t(X), method="dw")
    assert bool(torch.isnan(R3[1, 1, 1]))


def test_dw_residual_refuses_other_operators(bt):
    N, M = 16, 16
    A, B, C = gen.dominant_blocks(N, M, seed=1)
    F = np.zeros((N, M, 2))
    with bt.factor(_t(A), _t(B), _t(C), 4) as fac:
        with pytest.raises(bt.BtError) as ei:
            fac.residual(_t(F), _t(F), method="dw")
        assert ei.value.name == "BT_ERR_UNSUPPORTED"
    # a stencil whose off-diagonals are not -1
    A, B, C = gen.acoustic_system(N, M)
    idx = np.arange(M - 1)
    C[:, idx, idx + 1] = -0.5
    with bt.factor(_t(A), _t(B), _t(C), 4) as fac:
        assert fac.stencil == 1
        with pytest.raises(bt.BtError) as ei:
            fac.residual(_t(F), _t(F), method="dw")
        assert ei.value.name == "BT_ERR_UNSUPPORTED"
        # the refinement then forms its residual in FP64 and still converges
        Fr = gen.uniform_rhs(N, M, 3, seed=2)
        X, info = fac.solve(_t(Fr), precision="f32", tol=1e-12, return_info=True)
    assert info["converged"]
    assert oracle.rel_res(A, B, C, X.cpu().numpy(), Fr) <= 2e-12
    # M not a multiple of 8
    A, B, C = gen.acoustic_system(N, 12)
    with bt.factor(_t(A), _t(B), _t(C), 4) as fac:
        with pytest.raises(bt.BtError) as ei:
            fac.residual(_t(np.zeros((N, 12, 1))), _t(np.zeros((N, 12, 1))), method="dw")
        assert ei.value.name == "BT_ERR_UNSUPPORTED"


@pytest.mark.parametrize("prec", ["bf16x3", "f32"])
def test_refinement_with_dw_and_fp64_residuals_agree(bt, prec):
    N, M, K, S = 64, 128, 40, 8
    A, B, C = gen.acoustic_system(N, M)
    F = gen.acoustic_rhs(N, M, K, seed=12)
    Xr = oracle.solve_block_thomas(A, B, C, F)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        out = {}
        for res in ("dw", "fp64"):
            X, info = fac.solve(_t(F), precision=prec, tol=1e-12, residual=res, return_info=True)
            assert info["converged"], (res, info)
            out[res] = X.cpu().numpy()
    for res, X in out.items():
        assert oracle.rel_res(A, B, C, X, F) <= 2e-12, res
        assert oracle.rel_err(X, Xr) <= 1e-10, res
        assert oracle.col_err(X, Xr) <= 1e-10, res


def test_refinement_with_out_of_range_values(bt):
    # F scaled by 2^80: every residual of the refinement falls back to FP64
    N, M, K, S = 32, 64, 8, 4
    A, B, C = gen.acoustic_system(N, M)
    F = gen.acoustic_rhs(N, M, K, seed=13) * 2.0 ** 80
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        X, info = fac.solve(_t(F), precision="bf16x3", tol=1e-12, residual="dw", return_info=True)
    X = X.cpu().numpy()
    assert info["converged"]
    assert oracle.rel_res(A, B, C, X, F) <= 2e-12
    assert oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-10
    assert oracle.col_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-10
