"""Schur-complement CG with a probing band preconditioner on the GPU (Section 3.3)
against the oracle: each step (product with S, reduced right-hand side, the
probed band matrix) element by element, and the whole solve against the direct
block-tridiagonal solve of the grid (GPU only)."""

import numpy as np
import pytest

import oracle
from oracle import schur

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


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# (nr, h, p, shift, S): several strips, a strip of one row, M = 64 strips
SHAPES = [(64, 8, 3, 0.0, 8), (40, 5, 4, 0.25, 4), (33, 1, 2, 1.0, 3), (96, 64, 2, 0.0, 8)]


@pytest.mark.parametrize("nr,h,p,shift,S", SHAPES)
def test_schur_product_and_rhs(bt, nr, h, p, shift, S):
    K = 3
    rng = np.random.default_rng(nr + h)
    v = rng.uniform(-1, 1, (p - 1, nr, K))
    nz = p * h + p - 1
    F = rng.uniform(-1, 1, (nz, nr, K))
    with bt.SchurPCG(nr, h, p, shift, d=-1, S=S) as sp:
        assert (sp.nz, sp.ng) == (nz, (p - 1) * nr)
        Sv = sp.apply(_t(v)).cpu().numpy()
        g = sp.rhs(_t(F)).cpu().numpy()
    assert _rel(Sv, schur.schur_apply(v, nr, h, p, shift)) <= 1e-12
    assert _rel(g, schur.schur_rhs(F, nr, h, p, shift)) <= 1e-12


@pytest.mark.parametrize("d", [0, 3, 9])
def test_probed_band(bt, d):
    nr, h, p, shift, S = 40, 5, 4, 0.25, 4
    n = (p - 1) * nr
    SP = schur.schur_apply(schur.probing_vectors(n, d).reshape(p - 1, nr, -1), nr, h, p, shift).reshape(n, -1)
    ab_ref = schur.probe_band(SP, d)
    with bt.SchurPCG(nr, h, p, shift, d=d, S=S) as sp:
        ab = sp.band().cpu().numpy()
        assert sp.band_M >= max(d, 16)
    assert _rel(ab, ab_ref) <= 1e-12


@pytest.mark.parametrize("d", [-1, 0, 2, 6])
@pytest.mark.parametrize("K", [1, 5])
def test_schur_solve(bt, d, K):
    nr, h, p, shift, S = 64, 8, 3, 0.0, 8
    nz = p * h + p - 1
    F = np.random.default_rng(K).uniform(-1, 1, (nz, nr, K))
    with bt.SchurPCG(nr, h, p, shift, d=d, S=S) as sp:
        X, info = sp.solve(_t(F), tol=1e-11, return_info=True)
    X = X.cpu().numpy()
    A, B, C = schur.grid_blocks(nr, nz, shift)
    assert info["converged"] and info["rel_res"] <= 1e-11
    assert oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-9
    assert oracle.col_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-9
    # iteration count of the oracle's PCG with the oracle's S and B
    n = (p - 1) * nr
    g = schur.schur_rhs(F, nr, h, p, shift).reshape(n, K)
    apply = lambda u: schur.schur_apply(u.reshape(p - 1, nr, -1), nr, h, p, shift).reshape(n, -1)  # noqa: E731
    if d < 0:
        solve_B = lambda r: r.copy()  # noqa: E731
    else:
        Bm = oracle.band_dense(schur.probe_band(apply(schur.probing_vectors(n, d)), d), d, d)
        solve_B = lambda r: np.linalg.solve(Bm, r)  # noqa: E731
    _, it_ref, _ = schur.pcg(apply, solve_B, g, 1e-11, 1000)
    assert abs(info["iters"] - it_ref) <= 1, (info["iters"], it_ref)


def test_schur_solve_larger_grid_residual(bt):
    # 4 strips of 64 rows, 1024 columns (259 x 1024 grid), 4 right-hand sides,
    # one of them zero: residual of the whole grid operator by its definition
    nr, h, p, shift, S, K = 1024, 64, 4, 0.0, 16, 4
    nz = p * h + p - 1
    F = np.random.default_rng(9).uniform(-1, 1, (nz, nr, K))
    F[:, :, 2] = 0.0
    its = {}
    for d in (-1, 8):
        with bt.SchurPCG(nr, h, p, shift, d=d, S=S) as sp:
            X, info = sp.solve(_t(F), tol=1e-10, return_info=True)
        X = X.cpu().numpy()
        assert info["converged"]
        R = F - schur.grid_apply(X, shift)
        assert np.sqrt((R ** 2).sum()) <= 1e-8 * np.sqrt((F ** 2).sum())
        assert (X[:, :, 2] == 0).all()
        its[d] = info["iters"]
    assert its[8] < its[-1], its


def test_schur_nonconvergence_and_arguments(bt):
    nr, h, p = 32, 4, 2
    F = _t(np.random.default_rng(1).uniform(-1, 1, (p * h + p - 1, nr, 2)))
    with bt.SchurPCG(nr, h, p, 0.0, d=1, S=4) as sp:
        with pytest.raises(bt.BtError) as e:
            sp.solve(F, tol=1e-15, max_it=1)
        assert e.value.name == "BT_ERR_NOCONV"
        X, info = sp.solve(F, tol=1e-15, max_it=1, return_info=True, check=False)
        assert info["iters"] == 1 and not info["converged"] and np.isfinite(X.cpu().numpy()).all()
        with pytest.raises(ValueError):
            sp.solve(F[:, :16])
        lib = bt._lib.load()
        P = bt.solver._ptr
        assert bt._lib.STATUS_NAMES[lib.bt_schur_solve(sp._h, P(F), 2, P(F), 1e-8, 10, None, None)] == "BT_ERR_ARG"
        assert bt._lib.STATUS_NAMES[lib.bt_schur_solve(sp._h, P(F), 2, P(F), 0.0, 10, None, None)] == "BT_ERR_ARG"
    with bt.SchurPCG(nr, h, p, 0.0, d=-1, S=4) as sp:  # no preconditioner: no band to copy
        st = bt._lib.load().bt_schur_band(sp._h, bt.solver._ptr(F))
        assert bt._lib.STATUS_NAMES[st] == "BT_ERR_ARG"
        with pytest.raises(ValueError):
            sp.band()
