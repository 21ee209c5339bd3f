"""Pins of the CPU oracle against facts fixed independently of its code.

Every oracle function is checked here against at least one of: a hand-typed
golden fixture, a closed form, a library routine (LAPACK dense LU, banded LU),
a defining identity, or brute force on a tiny input.  The mutation tests at the
end plant plausible mistakes in copies of oracle routines and check that the
pins catch them.
"""

import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import alg2 as alg2_mod
from oracle import blocktri
from workloads import gen


def _rand_system(N, M, K, seed):
    A, B, C = gen.dominant_blocks(N, M, seed)
    F = gen.uniform_rhs(N, M, K, seed + 7)
    return A, B, C, F


def _read_blocks(path):
    blocks, P = {}, []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "P":
                P.append([float(x) for x in tok[1:]])
            else:
                blocks[tok[0]] = np.array([float(x) for x in tok[1:]]).reshape(2, 2)
    A = np.stack([blocks[f"A{j}"] for j in (1, 2, 3)])
    B = np.stack([blocks[f"B{j}"] for j in (1, 2, 3)])
    C = np.stack([blocks[f"C{j}"] for j in (1, 2, 3)])
    return A, B, C, np.array(P)


# --------------------------------------------------------------------------
# eq. main-eq: layout, product, solutions
# --------------------------------------------------------------------------

def test_dense_P_matches_hand_typed_layout(golden_dir):
    A, B, C, P = _read_blocks(os.path.join(golden_dir, "main_eq_N3_M2.txt"))
    np.testing.assert_array_equal(oracle.dense_P(A, B, C), P)


def test_apply_P_matches_hand_typed_layout(golden_dir):
    A, B, C, P = _read_blocks(os.path.join(golden_dir, "main_eq_N3_M2.txt"))
    X = np.arange(12, dtype=float).reshape(3, 2, 2) - 5.0
    np.testing.assert_allclose(oracle.apply_P(A, B, C, X).reshape(6, 2), P @ X.reshape(6, 2), rtol=0, atol=0)


def test_apply_P_ignores_unused_corner_blocks():
    A, B, C, F = _rand_system(5, 3, 2, 11)
    A2, B2 = A.copy(), B.copy()
    A2[0] = 123.0
    B2[-1] = -77.0
    np.testing.assert_array_equal(oracle.apply_P(A, B, C, F), oracle.apply_P(A2, B2, C, F))


def test_scalar_green_function(golden_dir):
    N = 4
    A = np.ones((N, 1, 1)); B = np.ones((N, 1, 1)); C = 2.0 * np.ones((N, 1, 1))
    A[0] = 0; B[-1] = 0
    with open(os.path.join(golden_dir, "laplace1d_N4.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    for tok in rows:
        F = np.array([float(x) for x in tok[1:5]]).reshape(N, 1, 1)
        Xe = np.array([float(x) for x in tok[6:10]]).reshape(N, 1, 1)
        np.testing.assert_allclose(oracle.solve_block_thomas(A, B, C, F), Xe, rtol=0, atol=1e-15)
        np.testing.assert_allclose(oracle.solve_dense(A, B, C, F), Xe, rtol=0, atol=1e-15)


@pytest.mark.parametrize("N,M,K,seed", [(1, 3, 2, 0), (2, 1, 1, 1), (7, 3, 2, 2), (16, 4, 3, 3), (9, 8, 1, 4)])
def test_block_thomas_matches_lapack_dense_lu(N, M, K, seed):
    A, B, C, F = _rand_system(N, M, K, seed)
    Xd = np.linalg.solve(oracle.dense_P(A, B, C), F.reshape(N * M, K)).reshape(N, M, K)
    X = oracle.solve_block_thomas(A, B, C, F)
    assert oracle.rel_err(X, Xd) < 1e-14
    assert oracle.rel_res(A, B, C, X, F) < 1e-14


def test_scalar_case_matches_banded_lapack():
    # M = 1 is a tridiagonal system: LAPACK's banded LU (gbsv) is an independent routine.
    rng = np.random.default_rng(5)
    N = 50
    a = rng.random(N); b = rng.random(N); c = 3.0 + rng.random(N)
    a[0] = 0; b[-1] = 0
    f = rng.uniform(-1, 1, N)
    ab = np.zeros((3, N))
    ab[0, 1:] = -b[:-1]
    ab[1] = c
    ab[2, :-1] = -a[1:]
    x = scipy.linalg.solve_banded((1, 1), ab, f)
    X = oracle.solve_block_thomas(a.reshape(N, 1, 1), b.reshape(N, 1, 1), c.reshape(N, 1, 1), f.reshape(N, 1, 1))
    np.testing.assert_allclose(X.ravel(), x, rtol=1e-14, atol=1e-15)


def test_poisson_closed_form_separation_of_variables():
    # Five-point operator, manufactured solution from exact eigen-pairs of the
    # discrete Laplacian (separation of variables): X is known exactly.
    N, M, K = 48, 20, 4
    A, B, C = gen.poisson_system(N, M)
    X_exact, F = gen.poisson_manufactured(N, M, K, seed=3)
    X = oracle.solve_block_thomas(A, B, C, F)
    lam_min = 4 - 2 * math.cos(math.pi / (M + 1)) - 2 * math.cos(math.pi / (N + 1))
    kappa = 8.0 / lam_min
    assert oracle.rel_err(X, X_exact) < kappa * 1e-15
    assert oracle.rel_err(X, X_exact) < 1e-12


def test_poisson_closed_form_is_consistent_with_product():
    # The manufactured F must equal P X_exact (pins the generator used by the closed-form test).
    N, M, K = 12, 7, 3
    A, B, C = gen.poisson_system(N, M)
    X_exact, F = gen.poisson_manufactured(N, M, K, seed=9)
    np.testing.assert_allclose(oracle.apply_P(A, B, C, X_exact), F, rtol=0, atol=1e-13)


def test_residual_and_error_norms():
    A, B, C, F = _rand_system(10, 3, 2, 8)
    X = oracle.solve_dense(A, B, C, F)
    r = oracle.residual(A, B, C, X, F)
    assert np.abs(r).max() < 1e-13
    assert oracle.rel_err(2 * X, X) == pytest.approx(1.0)
    assert oracle.rel_res(A, B, C, np.zeros_like(F), F) == pytest.approx(1.0)
    # per-column error: each column measured against its own largest entry
    Xr = np.zeros((2, 2, 3))
    Xr[:, :, 0] = [[1.0, -4.0], [2.0, 0.5]]   # max |.| 4
    Xr[:, :, 1] = [[1e-6, 0.0], [0.0, 0.0]]   # max |.| 1e-6
    Xr[:, :, 2] = [[3.0, 3.0], [3.0, 3.0]]
    Xe = Xr.copy()
    Xe[0, 1, 0] += 0.4      # 0.4 / 4 = 0.1 in column 0
    Xe[1, 1, 1] += 2e-7     # 2e-7 / 1e-6 = 0.2 in column 1 (tiny against the panel's norm)
    assert oracle.col_err(Xe, Xr) == pytest.approx(0.2)
    assert oracle.rel_err(Xe, Xr) < 0.1


# --------------------------------------------------------------------------
# Section 2.2: segments, responses, reduced system, Algorithm 1, Algorithm 2
# --------------------------------------------------------------------------

def _schur(P, gamma):
    n = P.shape[0]
    inner = np.setdiff1d(np.arange(n), gamma)
    Pgg = P[np.ix_(gamma, gamma)]
    Pgi = P[np.ix_(gamma, inner)]
    Pig = P[np.ix_(inner, gamma)]
    Pii = P[np.ix_(inner, inner)]
    return Pgg - Pgi @ np.linalg.solve(Pii, Pig), Pgi, Pii, inner


@pytest.mark.parametrize("N,M,S", [(12, 3, 3), (16, 2, 4), (20, 4, 5), (8, 3, 8), (9, 2, 1)])
def test_reduced_system_is_schur_complement(N, M, S):
    # P~ of eq. red1 is the Schur complement of P onto the interface rows
    # (the same algebra as eq. schur_decomp); F~ likewise.
    A, B, C, F = _rand_system(N, M, 2, 20 + N)
    U, V = oracle.segment_responses(A, B, C, S)
    W = oracle.segment_W(A, B, C, F, S)
    At, Ct, Bt = oracle.reduced_system(A, B, C, S, U, V)
    Ft = oracle.reduced_rhs(A, B, F, W, S)
    L = N // S
    gamma = np.concatenate([np.arange(s * L * M, s * L * M + M) for s in range(S)])
    P = oracle.dense_P(A, B, C)
    Sg, Pgi, Pii, inner = _schur(P, gamma)
    Ptil = oracle.dense_P(At, Bt, Ct)
    np.testing.assert_allclose(Ptil, Sg, rtol=0, atol=1e-12 * np.abs(Sg).max())
    f = F.reshape(N * M, 2)
    ftil = f[gamma] - Pgi @ np.linalg.solve(Pii, f[inner])
    np.testing.assert_allclose(Ft.reshape(S * M, 2), ftil, rtol=0, atol=1e-12 * np.abs(ftil).max())


@pytest.mark.parametrize("N,M,S", [(12, 3, 3), (16, 2, 4), (15, 3, 5)])
def test_superposition_holds_for_true_solution(N, M, S):
    # eq. superposition: X_i = U_i X_K + V_i X_{K+L} + W_i with the exact X plugged in.
    A, B, C, F = _rand_system(N, M, 3, 40 + N)
    X = oracle.solve_dense(A, B, C, F)
    U, V = oracle.segment_responses(A, B, C, S)
    W = oracle.segment_W(A, B, C, F, S)
    L = N // S
    for s, (k, a, b) in enumerate(oracle.segment_rows(N, S)):
        right = X[k + L] if k + L < N else np.zeros_like(X[0])
        for i in range(a, b):
            np.testing.assert_allclose(U[i] @ X[k] + V[i] @ right + W[i], X[i], rtol=0, atol=1e-13)


def test_responses_satisfy_their_subproblems():
    # eqs. sub1-sub3 row by row, including the boundary data.
    N, M, S = 15, 3, 3
    A, B, C, F = _rand_system(N, M, 2, 77)
    U, V = oracle.segment_responses(A, B, C, S)
    W = oracle.segment_W(A, B, C, F, S)
    L = N // S
    I = np.eye(M)
    for k, a, b in oracle.segment_rows(N, S):
        ext_U = {k: I, k + L: np.zeros((M, M))}
        ext_V = {k: np.zeros((M, M)), k + L: I}
        ext_W = {k: np.zeros((M, 2)), k + L: np.zeros((M, 2))}
        for i in range(a, b):
            def val(Z, ext, r):
                return ext[r] if r in ext else Z[r]
            bi = B[i] if i < N - 1 else np.zeros((M, M))
            for Z, ext, rhs in ((U, ext_U, 0.0), (V, ext_V, 0.0), (W, ext_W, F[i])):
                lhs = -A[i] @ val(Z, ext, i - 1) + C[i] @ Z[i] - bi @ val(Z, ext, i + 1)
                np.testing.assert_allclose(lhs, rhs + 0 * lhs, rtol=0, atol=1e-13)


@pytest.mark.parametrize("S", [1, 2, 3, 5, 7, 8, 16])
def test_dichotomy_matches_dense_solve_of_reduced_system(S):
    rng = np.random.default_rng(S)
    M, K = 3, 2
    At = rng.random((S, M, M)); Bt = rng.random((S, M, M)); Ct = rng.random((S, M, M)) + 8 * np.eye(M)
    At[0] = 0; Bt[-1] = 0
    Ft = rng.uniform(-1, 1, (S, M, K))
    Xt = oracle.dichotomy_solve(At, Ct, Bt, Ft)
    ref = np.linalg.solve(oracle.dense_P(At, Bt, Ct), Ft.reshape(S * M, K)).reshape(S, M, K)
    np.testing.assert_allclose(Xt, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("S", [1, 4, 6, 9])
def test_dichotomy_tree_rows_are_inverse_rows(S):
    # Defining property of step 1 of Algorithm 1: the stored block row R_{m,.}
    # times the node's sub-matrix {P~}_l^r is the m-th unit block row.
    rng = np.random.default_rng(100 + S)
    M = 2
    At = rng.random((S, M, M)); Bt = rng.random((S, M, M)); Ct = rng.random((S, M, M)) + 6 * np.eye(M)
    At[0] = 0; Bt[-1] = 0
    nodes = oracle.dichotomy_tree(At, Ct, Bt)
    covered = sorted(n.m for n in nodes)
    assert covered == list(range(S))  # every unknown is the middle of exactly one node
    depth = max(n.level for n in nodes) + 1
    assert depth == math.ceil(math.log2(S + 1))
    for n in nodes:
        sub = oracle.dense_P(At[n.l:n.r + 1].copy(), Bt[n.l:n.r + 1].copy(), Ct[n.l:n.r + 1].copy())
        row = np.concatenate(list(n.R), axis=1)
        e = np.zeros_like(row)
        e[:, (n.m - n.l) * M:(n.m - n.l + 1) * M] = np.eye(M)
        np.testing.assert_allclose(row @ sub, e, rtol=0, atol=1e-13)
        if n.l > 0:
            np.testing.assert_allclose(n.HL, n.R[0] @ At[n.l], atol=0)
        if n.r < S - 1:
            np.testing.assert_allclose(n.HR, n.R[-1] @ Bt[n.r], atol=0)


@pytest.mark.parametrize("N,M,K,S", [(64, 4, 1, 8), (24, 3, 2, 1), (24, 3, 2, 2), (24, 3, 2, 6), (24, 3, 2, 24), (30, 2, 3, 5)])
def test_alg2_matches_dense_lu(N, M, K, S):
    A, B, C, F = _rand_system(N, M, K, N + S)
    X = oracle.alg2_solve(A, B, C, F, S)
    Xd = oracle.solve_dense(A, B, C, F)
    assert oracle.rel_err(X, Xd) < 1e-13


def test_alg2_single_segment_is_block_thomas():
    # S = 1: one interface (row 1) and one segment -- the method reduces to the
    # block sweep of the whole system.
    A, B, C, F = _rand_system(40, 4, 3, 5)
    X1 = oracle.alg2_solve(A, B, C, F, 1)
    Xt = oracle.solve_block_thomas(A, B, C, F)
    assert oracle.rel_err(X1, Xt) < 1e-14


def test_alg2_all_interfaces_reduces_to_algorithm1_on_P():
    # S = N (L = 1): P~ is P itself and the dichotomy is Algorithm 1 on the full system.
    N, M = 10, 3
    A, B, C, F = _rand_system(N, M, 2, 6)
    U, V = oracle.segment_responses(A, B, C, N)
    At, Ct, Bt = oracle.reduced_system(A, B, C, N, U, V)
    np.testing.assert_array_equal(Ct, C)
    np.testing.assert_array_equal(At[1:], A[1:])
    np.testing.assert_array_equal(Bt[:-1], B[:-1])
    Xd = oracle.dichotomy_solve(At, Ct, Bt, F)
    assert oracle.rel_err(Xd, oracle.solve_dense(A, B, C, F)) < 1e-14


def test_segment_rows_require_divisibility():
    with pytest.raises(ValueError):
        oracle.segment_rows(10, 3)
    assert oracle.segment_rows(6, 3) == [(0, 1, 2), (2, 3, 4), (4, 5, 6)]


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------

def test_transpose_blocks_is_matrix_transpose():
    A, B, C, F = _rand_system(6, 3, 1, 9)
    np.testing.assert_array_equal(oracle.dense_P(*oracle.transpose_blocks(A, B, C)), oracle.dense_P(A, B, C).T)


def test_adjoint_dot_product_identity():
    A, B, C, F = _rand_system(12, 3, 2, 12)
    G = gen.uniform_rhs(12, 3, 2, 99)
    X = oracle.solve_block_thomas(A, B, C, F)
    lam = oracle.solve_block_thomas(*oracle.transpose_blocks(A, B, C), G)
    assert np.vdot(G, X) == pytest.approx(np.vdot(lam, F), rel=1e-13)


def test_adjoint_gradients_match_central_differences():
    # L = 0.5 ||X - X_t||^2, central differences in FP64 with h = 1e-6 on N=16, M=4, K=2.
    # L(+h) - L(-h) is evaluated as 0.5 * sum((X+ - X-) * (X+ + X- - 2 X_t)), an
    # exact rewriting that avoids cancelling two nearly equal losses.
    N, M, K = 16, 4, 2
    A, B, C, F = _rand_system(N, M, K, 13)
    Xt = gen.uniform_rhs(N, M, K, 14)
    X = oracle.solve_block_thomas(A, B, C, F)
    dF, dA, dB, dC = oracle.adjoint_grads(A, B, C, X, X - Xt)
    h = 1e-6
    rng = np.random.default_rng(0)
    checks = 0
    for name, arr, grad in (("F", F, dF), ("A", A, dA), ("B", B, dB), ("C", C, dC)):
        for _ in range(12):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            if name == "A" and idx[0] == 0 or name == "B" and idx[0] == N - 1:
                assert grad[idx] == 0.0
                continue
            args = {"A": A, "B": B, "C": C, "F": F}
            plus = {k: v.copy() for k, v in args.items()}
            minus = {k: v.copy() for k, v in args.items()}
            plus[name][idx] += h
            minus[name][idx] -= h
            Xp = oracle.solve_dense(plus["A"], plus["B"], plus["C"], plus["F"])
            Xm = oracle.solve_dense(minus["A"], minus["B"], minus["C"], minus["F"])
            fd = 0.5 * float(np.sum((Xp - Xm) * (Xp + Xm - 2 * Xt))) / (2 * h)
            assert fd == pytest.approx(grad[idx], rel=1e-6, abs=1e-12)
            checks += 1
    assert checks >= 40


# --------------------------------------------------------------------------
# generators
# --------------------------------------------------------------------------

def test_dominant_blocks_are_strictly_diagonally_dominant():
    A, B, C = gen.dominant_blocks(10, 5, 0)
    assert np.all(A[0] == 0) and np.all(B[-1] == 0)
    idx = np.arange(5)
    d = C[:, idx, idx]
    off = np.abs(A).sum(2) + np.abs(B).sum(2) + np.abs(C).sum(2) - np.abs(d)
    assert np.all(d - off >= 1.0) and np.all(d - off < 2.0)
    assert A.min() >= 0 and A.max() < 1 and np.abs(C - np.where(np.eye(5, dtype=bool), C, 0)).max() <= 0.5


def test_pml_profile_values():
    s = gen.pml_sigma(100)
    assert s[0] == pytest.approx(2.0) and s[-1] == pytest.approx(2.0)
    assert s[19] == pytest.approx(2.0 * (1 / 20) ** 2) and s[20] == 0.0 and s[79] == 0.0
    np.testing.assert_allclose(s, s[::-1])


def test_generators_regenerate_column_subsets():
    F = gen.acoustic_rhs(8, 6, 5, seed=3)
    np.testing.assert_array_equal(gen.acoustic_rhs(8, 6, 5, seed=3, columns=[1, 4]), F[:, :, [1, 4]])
    X, F2 = gen.poisson_manufactured(9, 4, 6, seed=2)
    X2, F3 = gen.poisson_manufactured(9, 4, 6, seed=2, columns=[5])
    np.testing.assert_array_equal(X2[:, :, 0], X[:, :, 5])
    assert gen.source_wavelet(np.array([0.2]))[0] == 0.0


def test_batched_K_distribution():
    Ks = gen.batched_K(64, 5)
    assert len(Ks) == 64 and min(Ks) >= 1 and max(Ks) <= 1024


# --------------------------------------------------------------------------
# mutation checks: plausible mistakes planted in copies of oracle routines
# --------------------------------------------------------------------------

def _thomas_mutant(kind):
    def solve(A, B, C, F):
        N, M, K = F.shape
        alpha = np.empty((N, M, M)); beta = np.empty((N, M, K))
        for j in range(N):
            if j == 0:
                D, rhs = C[0], F[0]
            else:
                Aj = A[j].T if kind == "transpose" else A[j]
                D = C[j] - (Aj @ alpha[j - 1] if kind != "drop_term" else 0)
                sgn = -1.0 if kind == "sign" else 1.0
                rhs = F[j] + sgn * Aj @ beta[j - 1]
            sol = np.linalg.solve(D, np.concatenate([B[j], rhs], axis=1))
            alpha[j], beta[j] = sol[:, :M], sol[:, M:]
        X = np.empty_like(beta); X[-1] = beta[-1]
        for j in range(N - 2, -1, -1):
            nxt = j + 2 if (kind == "index" and j + 2 < N) else j + 1
            X[j] = beta[j] + alpha[j] @ X[nxt]
        return X
    return solve


@pytest.mark.parametrize("kind", ["transpose", "drop_term", "sign", "index"])
def test_pins_catch_planted_thomas_mistakes(kind):
    A, B, C, F = _rand_system(9, 3, 2, 3)
    Xd = np.linalg.solve(oracle.dense_P(A, B, C), F.reshape(27, 2)).reshape(9, 3, 2)
    assert oracle.rel_err(_thomas_mutant(kind)(A, B, C, F), Xd) > 1e-6


def test_pins_catch_planted_reduced_system_mistake(monkeypatch):
    # Flip the sign of the A_K V_{K-1} term of eq. red1: the Schur-complement pin must fail.
    N, M, S = 12, 3, 3
    A, B, C, F = _rand_system(N, M, 2, 32)
    U, V = oracle.segment_responses(A, B, C, S)
    At, Ct, Bt = oracle.reduced_system(A, B, C, S, U, V)
    L = N // S
    Ct_bad = Ct.copy()
    for s in range(1, S):
        Ct_bad[s] = Ct[s] + 2 * A[s * L] @ V[s * L - 1]
    gamma = np.concatenate([np.arange(s * L * M, s * L * M + M) for s in range(S)])
    Sg = _schur(oracle.dense_P(A, B, C), gamma)[0]
    assert np.abs(oracle.dense_P(At, Bt, Ct) - Sg).max() < 1e-12
    assert np.abs(oracle.dense_P(At, Bt, Ct_bad) - Sg).max() > 1e-6


def test_pins_catch_planted_dichotomy_mistake():
    # A copy of Algorithm 1 whose right-half update uses At_m instead of At_{m+1}
    # (an index slip in eq. subb): the dense pin must reject it.
    S, M, K = 7, 2, 1
    rng = np.random.default_rng(1)
    At = rng.random((S, M, M)); Bt = rng.random((S, M, M)); Ct = rng.random((S, M, M)) + 5 * np.eye(M)
    At[0] = 0; Bt[-1] = 0
    Ft = rng.uniform(-1, 1, (S, M, K))
    ref = np.linalg.solve(oracle.dense_P(At, Bt, Ct), Ft.reshape(S * M, K)).reshape(S, M, K)
    nodes = {(n.l, n.r): n for n in oracle.dichotomy_tree(At, Ct, Bt)}

    def mutant():
        X = np.zeros((S, M, K))
        work = [(0, S - 1, Ft.copy())]
        while work:
            l, r, rhs = work.pop(0)
            if l > r:
                continue
            n = nodes[(l, r)]
            X[n.m] = np.einsum("tab,tbk->ak", n.R, rhs[l:r + 1])
            if l <= n.m - 1:
                left = rhs.copy(); left[n.m - 1] += Bt[n.m - 1] @ X[n.m]
                work.append((l, n.m - 1, left))
            if n.m + 1 <= r:
                right = rhs.copy(); right[n.m + 1] += At[n.m] @ X[n.m]
                work.append((n.m + 1, r, right))
        return X

    assert np.abs(oracle.dichotomy_solve(At, Ct, Bt, Ft) - ref).max() < 1e-13
    assert np.abs(mutant() - ref).max() > 1e-6


# ---------------------------------------------------------------------------
# band matrices as block-tridiagonal systems (Section 3.3.1, item c)
# ---------------------------------------------------------------------------
from oracle import band as band_mod  # noqa: E402
import scipy.sparse  # noqa: E402


@pytest.mark.parametrize("n,kl,ku", [(11, 2, 3), (40, 0, 4), (33, 5, 0), (17, 1, 1), (6, 5, 5)])
def test_band_dense_matches_scipy_dia(n, kl, ku):
    # SciPy's DIA format stores diagonal `offset` column-aligned, the same
    # convention as LAPACK band storage: an independent reading of ab
    ab = gen.band_matrix(n, kl, ku, seed=n)
    D = scipy.sparse.dia_matrix((ab, list(range(ku, -kl - 1, -1))), shape=(n, n)).toarray()
    assert np.array_equal(band_mod.band_dense(ab, kl, ku), D)


BAND_CASES = [(64, 8, 8, 8, 2, 2), (61, 3, 7, 8, 2, 3), (100, 12, 5, 16, 3, 1), (29, 1, 1, 1, 4, 2),
              (50, 0, 6, 6, 3, 2), (45, 9, 9, 9, 5, 1)]


@pytest.mark.parametrize("n,kl,ku,M,S,K", BAND_CASES)
def test_band_blocks_solve_matches_lapack_banded(n, kl, ku, M, S, K):
    # the block form, solved by block Thomas, against LAPACK's banded LU (gbsv)
    ab = gen.band_matrix(n, kl, ku, seed=n + M)
    F = np.random.default_rng(n).uniform(-1, 1, (n, K))
    A, B, C, N = band_mod.band_blocks(ab, kl, ku, M, S)
    assert N % S == 0 and N * M >= n and (N - S) * M < n  # fewest block rows S allows
    X = oracle.solve_block_thomas(A, B, C, band_mod.pad_rows(F, N, M)).reshape(N * M, K)
    Xl = scipy.linalg.solve_banded((kl, ku), ab, F)
    assert oracle.rel_err(X[:n], Xl) < 1e-13
    assert np.abs(X[n:]).max(initial=0.0) == 0.0  # identity rows, zero right-hand side


@pytest.mark.parametrize("n,kl,ku,M,S,K", BAND_CASES)
def test_band_blocks_product_and_triangular_structure(n, kl, ku, M, S, K):
    ab = gen.band_matrix(n, kl, ku, seed=n + M)
    X = np.random.default_rng(n + 1).uniform(-1, 1, (n, K))
    A, B, C, N = band_mod.band_blocks(ab, kl, ku, M, S)
    Q = scipy.sparse.dia_matrix((ab, list(range(ku, -kl - 1, -1))), shape=(n, n)).toarray()
    Y = oracle.apply_P(A, B, C, band_mod.pad_rows(X, N, M)).reshape(N * M, K)
    np.testing.assert_allclose(Y[:n], Q @ X, rtol=0, atol=1e-13 * np.abs(Q).sum(axis=1).max())
    # the structure the paper notes: A_j upper triangular (nonzero only where
    # c - r >= M - kl), B_j lower triangular (c - r <= ku - M)
    d = np.arange(M)[None, :] - np.arange(M)[:, None]
    assert (A[:, d < M - kl] == 0).all() and (B[:, d > ku - M] == 0).all()


def test_band_mutations_are_caught():
    n, kl, ku, M, S = 61, 3, 7, 8, 2
    ab = gen.band_matrix(n, kl, ku, seed=4)
    F = np.random.default_rng(4).uniform(-1, 1, (n, 2))
    Xl = scipy.linalg.solve_banded((kl, ku), ab, F)
    D = scipy.sparse.dia_matrix((ab, list(range(ku, -kl - 1, -1))), shape=(n, n)).toarray()
    # storage read transposed (ab[ku + j - i, i]): the DIA pin fails
    Qt = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - ku), min(n, i + kl + 1)):
            Qt[i, j] = ab[ku + j - i, i] if 0 <= ku + j - i <= kl + ku else 0.0
    assert not np.array_equal(Qt, D)
    # sign slip on the coupling blocks (A_j = +Q[jM.., (j-1)M..]): the gbsv pin fails
    A, B, C, N = band_mod.band_blocks(ab, kl, ku, M, S)
    X = oracle.solve_block_thomas(-A, B, C, band_mod.pad_rows(F, N, M)).reshape(N * M, 2)
    assert oracle.rel_err(X[:n], Xl) > 1e-6
    # off-by-one block row in the cut: the gbsv pin fails
    X = oracle.solve_block_thomas(np.roll(A, 1, axis=0), B, C, band_mod.pad_rows(F, N, M)).reshape(N * M, 2)
    assert oracle.rel_err(X[:n], Xl) > 1e-6
