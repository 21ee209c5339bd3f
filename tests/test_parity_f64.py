"""FP64 CUDA path vs the CPU oracle, element by element (GPU only).

Bar: relative error <= 1e-12 against the FP64 oracle (Frobenius over the
panel), the accuracy the plain FP64 method must reach.  Sizes span several
column tiles and a ragged last tile; the named workloads run at full size with
the oracle evaluated on sampled columns.
"""

import numpy as np
import pytest

import oracle
from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def bt():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1108_4181_gb300 as bt

    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    return bt


DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _solve(bt, A, B, C, F, S, **kw):
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        return fac.solve(_t(F), **kw).cpu().numpy()


def test_config0_tiny_random(bt):
    w = gen.config0()
    X = _solve(bt, w.A, w.B, w.C, w.F, w.S)
    Xr = oracle.solve_block_thomas(w.A, w.B, w.C, w.F)
    assert oracle.rel_err(X, Xr) <= TOL
    assert oracle.col_err(X, Xr) <= TOL
    assert oracle.rel_err(X, oracle.solve_dense(w.A, w.B, w.C, w.F)) <= TOL
    assert oracle.col_err(X, oracle.solve_dense(w.A, w.B, w.C, w.F)) <= TOL
    assert oracle.rel_res(w.A, w.B, w.C, X, w.F) <= TOL


@pytest.mark.parametrize("N,M,K,S", [
    (64, 4, 1, 1),      # S = 1: one segment, block sweep
    (64, 4, 3, 64),     # S = N: every row an interface (Algorithm 1 on P)
    (60, 5, 7, 6),      # odd M, ragged K
    (96, 12, 9, 12),    # several column tiles plus a ragged one
    (48, 33, 2, 4),     # M not a multiple of the warp
    (128, 16, 17, 32),  # L = 4
    (40, 8, 5, 20),     # L = 2: one interior row per segment
    (7, 3, 2, 7),       # odd S, all interfaces
    (30, 6, 4, 5),      # odd depth tree
])
def test_random_shapes(bt, N, M, K, S):
    A, B, C = gen.dominant_blocks(N, M, seed=N * 7 + M)
    F = gen.uniform_rhs(N, M, K, seed=K + 3)
    X = _solve(bt, A, B, C, F, S)
    assert oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, F)) <= TOL
    assert oracle.col_err(X, oracle.solve_block_thomas(A, B, C, F)) <= TOL


@pytest.mark.parametrize("N,M,S", [(256, 60, 64), (128, 150, 32), (2048, 60, 256)])
def test_paper_block_sizes(bt, N, M, S):
    # the block sizes of the paper's Tables 1-2 (M = 60, 150; not multiples of
    # the tensor-core tile), one right-hand side as there and a 256-column panel;
    # the last case at the tables' smallest N = 2^11, matrices drawn on the device
    # as the paper-shape bench draws them
    if N <= 256:
        A, B, C = gen.dominant_blocks(N, M, seed=N + M)
    else:
        A, B, C = (t.cpu().numpy() for t in gen.dominant_blocks_device(N, M, 1000 + N + M, DEV))
    for K in (1, 256):
        F = gen.uniform_rhs(N, M, K, seed=K)
        X = _solve(bt, A, B, C, F, S)
        assert oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, F)) <= TOL
        assert oracle.col_err(X, oracle.solve_block_thomas(A, B, C, F)) <= TOL
        assert oracle.rel_res(A, B, C, X, F) <= TOL


@pytest.mark.parametrize("M,scaled", [(128, False), (128, True), (120, True)])
def test_dense_factor_products_scaled_unknowns(bt, M, scaled):
    # dense M = 128 blocks: the factorisation's block products run on the
    # tensor cores as exact digit-slice sums (M = 120: FP64 products, the same
    # bar).  The scaled case multiplies the unknowns by powers of two spread
    # over 2^-200 .. 2^200 (A_j D, B_j D, C_j D), so the rows and columns of
    # every product span a wide exponent range; couplings with zero rows and
    # columns give products with all-zero rows or columns.  The solution of
    # the scaled system is D^-1 X.
    N, K, S = 256, 9, 8
    A, B, C = gen.dominant_blocks(N, M, seed=M)
    A[:, :5, :] = 0.0  # couplings only: C_j is the dominant diagonal block
    B[:, :, 3] = 0.0
    F = gen.uniform_rhs(N, M, K, seed=12)
    d = np.ones(M)
    if scaled:
        d = np.exp2(np.random.default_rng(5).integers(-200, 201, M)).astype(np.float64)
    As, Bs, Cs = A * d, B * d, C * d
    Xr = oracle.solve_block_thomas(A, B, C, F)
    with bt.factor(_t(As), _t(Bs), _t(Cs), S) as fac:
        X = fac.solve(_t(F)).cpu().numpy() * d[None, :, None]
        if not scaled:
            U, V = oracle.segment_responses(A, B, C, S)
            At, Ct, Bt = oracle.reduced_system(A, B, C, S, U, V)
            for name, ref in (("U", U), ("V", V), ("At", At), ("Ct", Ct), ("Bt", Bt)):
                got = fac.export(name).cpu().numpy()
                np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()), err_msg=name)
    assert oracle.rel_err(X, Xr) <= TOL
    assert oracle.col_err(X, Xr) <= TOL


@pytest.mark.parametrize("N,M,S", [(16, 256, 4), (12, 200, 3), (64, 200, 16)])
def test_large_block_sizes(bt, N, M, S):
    # pivot blocks up to M = 256 (8 rows per lane in the cluster inversion,
    # clusters of 4 or 8 CTAs for the small batches); M = 200: rows not a
    # multiple of the warp
    A, B, C = gen.dominant_blocks(N, M, seed=N + M)
    F = gen.uniform_rhs(N, M, 3, seed=5)
    X = _solve(bt, A, B, C, F, S)
    Xr = oracle.solve_block_thomas(A, B, C, F)
    assert oracle.rel_err(X, Xr) <= TOL
    assert oracle.col_err(X, Xr) <= TOL


def test_unused_corner_blocks_are_ignored(bt):
    N, M, K, S = 32, 4, 2, 4
    A, B, C = gen.dominant_blocks(N, M, seed=3)
    F = gen.uniform_rhs(N, M, K, seed=4)
    A2, B2 = A.copy(), B.copy()
    A2[0] = 1e6
    B2[-1] = -1e6
    np.testing.assert_array_equal(_solve(bt, A, B, C, F, S), _solve(bt, A2, B2, C, F, S))


def test_factor_exports_match_oracle_definitions(bt):
    N, M, S = 48, 6, 6
    A, B, C = gen.dominant_blocks(N, M, seed=21)
    U, V = oracle.segment_responses(A, B, C, S)
    At, Ct, Bt = oracle.reduced_system(A, B, C, S, U, V)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        assert fac.depth == 3 and fac.S == S and fac.stencil == 0
        for name, ref in (("U", U), ("V", V), ("At", At), ("Ct", Ct), ("Bt", Bt)):
            got = fac.export(name).cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()), err_msg=name)


def test_steps_match_oracle_intermediates(bt):
    # step 2.1 leaves W (eq. sub3) on interior rows, step 2.2 X~ (eq. red1) on interface rows
    N, M, K, S = 48, 5, 6, 8
    A, B, C = gen.dominant_blocks(N, M, seed=5)
    F = gen.uniform_rhs(N, M, K, seed=6)
    W = oracle.segment_W(A, B, C, F, S)
    Xr = oracle.solve_dense(A, B, C, F)
    L = N // S
    iface = np.arange(0, N, L)
    interior = np.setdiff1d(np.arange(N), iface)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        X1 = fac.solve_stages(_t(F), 1).cpu().numpy()
        np.testing.assert_allclose(X1[interior], W[interior], rtol=0, atol=1e-13)
        X2 = fac.solve_stages(_t(F), 2).cpu().numpy()
        np.testing.assert_allclose(X2[iface], Xr[iface], rtol=0, atol=1e-13)
        X3 = fac.solve_stages(_t(F), 3).cpu().numpy()
        np.testing.assert_array_equal(X3, fac.solve(_t(F)).cpu().numpy())


def test_stencil_detection(bt):
    A, B, C = gen.poisson_system(16, 8)
    with bt.factor(_t(A), _t(B), _t(C), 4) as fac:
        assert fac.stencil == 1


@pytest.mark.parametrize("M", [3, 64, 128])
def test_singular_pivot_is_reported(bt, M):
    # M = 3: one-CTA inversion; M = 64, 128: cluster inversions (4 pivot
    # blocks per launch: clusters of 4 and 8 CTAs)
    N, S = 16, 4
    A, B, C = gen.dominant_blocks(N, M, seed=1)
    C[5] = 0.0   # interior row of segment 1 with A_5 = B_5 = 0: D_5 singular
    A[5] = 0.0
    B[5] = 0.0
    with pytest.raises(bt.BtError) as ei:
        bt.factor(_t(A), _t(B), _t(C), S)
    assert ei.value.name == "BT_ERR_SINGULAR"


def test_argument_errors(bt):
    A, B, C = gen.dominant_blocks(12, 2, seed=1)
    with pytest.raises(bt.BtError) as ei:
        bt.factor(_t(A), _t(B), _t(C), 5)
    assert ei.value.name == "BT_ERR_ARG"
    with bt.factor(_t(A), _t(B), _t(C), 3) as fac:
        F = _t(gen.uniform_rhs(12, 2, 2, 1))
        with pytest.raises(bt.BtError):
            fac.solve(F, out=F)  # X aliases F


def test_host_buffers_end_to_end(bt):
    w = gen.config0()
    with bt.factor(_t(w.A), _t(w.B), _t(w.C), w.S) as fac:
        Xh = fac.solve(torch.from_numpy(w.F).pin_memory())
        assert Xh.device.type == "cpu"
        assert oracle.rel_err(Xh.numpy(), oracle.solve_block_thomas(w.A, w.B, w.C, w.F)) <= TOL
        assert oracle.col_err(Xh.numpy(), oracle.solve_block_thomas(w.A, w.B, w.C, w.F)) <= TOL


# ---------------------------------------------------------------------------
# named workloads at full size
# ---------------------------------------------------------------------------

def test_config1_poisson_full_size(bt):
    w = gen.config1()
    with bt.factor(_t(w.A), _t(w.B), _t(w.C), w.S) as fac:
        X = fac.solve(_t(w.F)).cpu().numpy()
    # closed form (separation of variables) for every column
    err_exact = oracle.rel_err(X, w.X_exact)
    cols = [0, 31, 63]
    Xr = oracle.solve_block_thomas(w.A, w.B, w.C, w.F[:, :, cols])
    err_oracle = oracle.rel_err(X[:, :, cols], Xr)
    assert err_oracle <= TOL, err_oracle
    assert oracle.col_err(X[:, :, cols], Xr) <= TOL
    assert err_exact <= 1e-11, err_exact  # kappa ~ 5e4 times FP64 rounding


def test_config2_acoustic_fp64_sampled_columns(bt):
    cols = [0, 130, 300, 511]  # one column in each 128-column tile
    w = gen.config2()
    with bt.factor(_t(w.A), _t(w.B), _t(w.C), w.S) as fac:
        X = fac.solve(_t(w.F)).cpu().numpy()
    Xr = oracle.solve_block_thomas(w.A, w.B, w.C, w.F[:, :, cols])
    assert oracle.rel_err(X[:, :, cols], Xr) <= TOL
    assert oracle.col_err(X[:, :, cols], Xr) <= TOL


def test_config4_matrix_fp64(bt):
    A, B, C, F, _ = gen.config4()
    cols = [0, 64, 127]
    with bt.factor(_t(A), _t(B), _t(C), 64) as fac:
        X = fac.solve(_t(F)).cpu().numpy()
    Xr = oracle.solve_block_thomas(A, B, C, F[:, :, cols])
    assert oracle.rel_err(X[:, :, cols], Xr) <= TOL
    assert oracle.col_err(X[:, :, cols], Xr) <= TOL


def test_left_responses_export_matches_definition(bt):
    # Y_i, the forward response of a segment interior to its left interface
    # value (Y_a = E_a, Y_i = E_i Y_{i-1}), is the last block of the solution
    # of the interior's leading principal subsystem (rows a..i) whose right-hand
    # side is A_a in its first block: forward elimination of rows a..i alone.
    N, M, S = 24, 5, 3
    L = N // S
    A, B, C = gen.dominant_blocks(N, M, seed=31)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        Y = fac.export("Y").cpu().numpy()
    for s in range(S):
        a = s * L + 1
        assert np.all(Y[s * L] == 0.0)
        for i in range(a, s * L + L):
            n = i - a + 1
            P = np.zeros((n * M, n * M))
            for r in range(n):
                P[r * M:(r + 1) * M, r * M:(r + 1) * M] = C[a + r]
                if r > 0:
                    P[r * M:(r + 1) * M, (r - 1) * M:r * M] = -A[a + r]
                if r + 1 < n:
                    P[r * M:(r + 1) * M, (r + 1) * M:(r + 2) * M] = -B[a + r]
            rhs = np.zeros((n * M, M))
            rhs[:M] = A[a]
            ref = np.linalg.solve(P, rhs)[(n - 1) * M:]
            np.testing.assert_allclose(Y[i], ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))
