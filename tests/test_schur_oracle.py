"""Pins of the oracle's Schur-complement CG (oracle/schur.py) against values fixed
independently of it: a sparse direct solve of the assembled five-point grid
operator (SciPy), the Schur complement assembled from index sets of that
matrix, band matrices that probing must reproduce exactly, and dense solves.
Planted mistakes in copies of the routines must fail the pins (CPU only)."""

import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.linalg

import oracle
from oracle import schur


def _grid_matrix(nz, nr, shift):
    """Five-point operator, grid row-major, assembled by Kronecker products."""
    def adj(n):
        return scipy.sparse.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1])
    return ((4.0 + shift) * scipy.sparse.identity(nz * nr) - scipy.sparse.kron(scipy.sparse.identity(nz), adj(nr))
            - scipy.sparse.kron(adj(nz), scipy.sparse.identity(nr))).tocsc()


def _dense_S_from_apply(nr, h, p, shift):
    n = (p - 1) * nr
    return schur.schur_apply(np.eye(n).reshape(p - 1, nr, n), nr, h, p, shift).reshape(n, n)


@pytest.mark.parametrize("nr,h,p,shift", [(12, 3, 3, 0.0), (9, 4, 2, 0.25), (7, 2, 4, 1.0)])
def test_schur_complement_matches_index_sets_of_the_grid_matrix(nr, h, p, shift):
    nz, strips, iface = schur.grid_rows(h, p)
    Ag = _grid_matrix(nz, nr, shift).toarray()
    G = np.concatenate([np.arange(z * nr, (z + 1) * nr) for z in iface])
    I = np.setdiff1d(np.arange(nz * nr), G)
    S_ref = Ag[np.ix_(G, G)] - Ag[np.ix_(G, I)] @ np.linalg.solve(Ag[np.ix_(I, I)], Ag[np.ix_(I, G)])
    S = _dense_S_from_apply(nr, h, p, shift)
    np.testing.assert_allclose(S, S_ref, rtol=0, atol=1e-13)
    np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-13)


@pytest.mark.parametrize("nr,h,p,shift", [(12, 3, 3, 0.0), (9, 4, 2, 0.25)])
def test_interface_system_and_recovery_match_the_direct_solve(nr, h, p, shift):
    nz, strips, iface = schur.grid_rows(h, p)
    K = 2
    F = np.random.default_rng(nr).uniform(-1, 1, (nz, nr, K))
    Xd = scipy.sparse.linalg.spsolve(_grid_matrix(nz, nr, shift), F.reshape(nz * nr, K)).reshape(nz, nr, K)
    g = schur.schur_rhs(F, nr, h, p, shift)
    S = _dense_S_from_apply(nr, h, p, shift)
    xG = np.linalg.solve(S, g.reshape(-1, K)).reshape(p - 1, nr, K)
    np.testing.assert_allclose(xG, Xd[iface], rtol=0, atol=1e-13)
    np.testing.assert_allclose(schur.recover(F, xG, nr, h, p, shift), Xd, rtol=0, atol=1e-13)
    # the grid operator in block form (rows as blocks) gives the same solution
    A, B, C = schur.grid_blocks(nr, nz, shift)
    np.testing.assert_allclose(oracle.solve_block_thomas(A, B, C, F), Xd, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n,d", [(37, 0), (37, 1), (37, 3), (20, 6), (5, 2)])
def test_probing_reproduces_symmetric_band_matrices(n, d):
    rng = np.random.default_rng(n + d)
    Bm = rng.uniform(-1, 1, (n, n))
    Bm = np.triu(np.tril(Bm + Bm.T, d), -d)
    ab = schur.probe_band(Bm @ schur.probing_vectors(n, d), d)
    np.testing.assert_allclose(oracle.band_dense(ab, d, d), Bm, rtol=0, atol=1e-14)


def test_probing_band_zero_gives_row_sums_and_symmetrises():
    rng = np.random.default_rng(1)
    S = rng.uniform(0, 1, (15, 15))
    ab = schur.probe_band(S @ schur.probing_vectors(15, 0), 0)
    np.testing.assert_allclose(ab[0], S.sum(axis=1), rtol=1e-14)
    Bm = np.triu(np.tril(rng.uniform(-1, 1, (15, 15)), 2), -2)  # not symmetric
    ab = schur.probe_band(Bm @ schur.probing_vectors(15, 2), 2)
    np.testing.assert_allclose(oracle.band_dense(ab, 2, 2), 0.5 * (Bm + Bm.T), rtol=0, atol=1e-15)


def _problem(nr=48, h=6, p=3, shift=0.0, K=3):
    nz, _, _ = schur.grid_rows(h, p)
    F = np.random.default_rng(3).uniform(-1, 1, (nz, nr, K))
    S = _dense_S_from_apply(nr, h, p, shift)
    g = schur.schur_rhs(F, nr, h, p, shift).reshape(-1, K)
    return S, g


def test_pcg_converges_to_the_dense_solution():
    S, g = _problem()
    x, it, rr = schur.pcg(lambda v: S @ v, lambda r: r.copy(), g, 1e-12, 500)
    assert (rr <= 1e-12).all() and it <= S.shape[0]
    np.testing.assert_allclose(x, np.linalg.solve(S, g), rtol=0, atol=1e-10 * np.abs(x).max())
    # an exact preconditioner converges in one step
    x1, it1, _ = schur.pcg(lambda v: S @ v, lambda r: np.linalg.solve(S, r), g, 1e-12, 50)
    assert it1 == 1
    np.testing.assert_allclose(x1, x, rtol=0, atol=1e-10 * np.abs(x).max())


def test_probing_preconditioner_cuts_iterations():
    S, g = _problem()
    n = S.shape[0]
    its = []
    for d in (0, 2, 6):
        ab = schur.probe_band(S @ schur.probing_vectors(n, d), d)
        Bm = oracle.band_dense(ab, d, d)
        _, it, rr = schur.pcg(lambda v: S @ v, lambda r: np.linalg.solve(Bm, r), g, 1e-10, 500)
        assert (rr <= 1e-10).all()
        its.append(it)
    _, it_none, _ = schur.pcg(lambda v: S @ v, lambda r: r.copy(), g, 1e-10, 500)
    # d = 0 probes with the all-ones vector: the diagonal of row sums, small
    # for this S (its rows nearly cancel), is a poor preconditioner; wider
    # bands cut the iterations below the unpreconditioned count
    assert its[2] < its[1] < it_none, (its, it_none)


def test_planted_mistakes_fail():
    nr, h, p, shift = 9, 4, 2, 0.25
    S = _dense_S_from_apply(nr, h, p, shift)
    nz, strips, iface = schur.grid_rows(h, p)
    Ag = _grid_matrix(nz, nr, shift).toarray()
    G = np.concatenate([np.arange(z * nr, (z + 1) * nr) for z in iface])
    I = np.setdiff1d(np.arange(nz * nr), G)
    # sign slip on the coupling term: S = A_GG + A_GI A_II^{-1} A_IG
    S_bad = Ag[np.ix_(G, G)] + Ag[np.ix_(G, I)] @ np.linalg.solve(Ag[np.ix_(I, I)], Ag[np.ix_(I, G)])
    assert np.abs(S - S_bad).max() > 1e-3
    # probing read transposed without symmetrisation on a non-symmetric band matrix
    Bm = np.triu(np.tril(np.random.default_rng(2).uniform(-1, 1, (11, 11)), 1), -1)
    SP = Bm @ schur.probing_vectors(11, 1)
    bad = np.zeros((3, 11))
    for j in range(11):
        for i in range(max(0, j - 1), min(11, j + 2)):
            bad[1 + i - j, j] = SP[j, i % 3]
    assert np.abs(bad - schur.probe_band(SP, 1)).max() > 1e-3
    # CG with the residual update's sign flipped does not converge
    S2, g = _problem(nr=24, h=4, p=2)
    x = np.zeros_like(g); r = g.copy(); pd = r.copy(); rz = (r * r).sum(0)
    for _ in range(60):
        q = S2 @ pd
        a = rz / (pd * q).sum(0)
        x += a * pd
        r += a * q  # planted
        rzn = (r * r).sum(0)
        pd = r + rzn / rz * pd
        rz = rzn
    assert np.abs(x - np.linalg.solve(S2, g)).max() > 1e-3


def test_grid_apply_matches_the_assembled_matrix():
    nz, nr, K = 11, 7, 3
    X = np.random.default_rng(5).uniform(-1, 1, (nz, nr, K))
    Y = _grid_matrix(nz, nr, 0.5) @ X.reshape(nz * nr, K)
    np.testing.assert_allclose(schur.grid_apply(X, 0.5), Y.reshape(nz, nr, K), rtol=0, atol=1e-14)
