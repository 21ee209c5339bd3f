"""Mixed-precision solve with FP64-residual iterative refinement vs the CPU oracle (GPU only).

Bars: the refined solution reaches the requested relative residual
||F - P X||_F / ||F||_F (measured by the oracle in FP64, independently of the
device's own report) and its error against the FP64 oracle is <= 1e-10.
"""

import numpy as np
import pytest

import oracle
from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
PRECISIONS = ["f32"]


@pytest.fixture(scope="module")
def bt():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1108_4181_gb300 as bt

    return bt


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("N,M,K,S", [(64, 4, 1, 8), (64, 8, 5, 8), (96, 33, 7, 12), (128, 64, 20, 16)])
def test_refined_dense_random(bt, prec, N, M, K, S):
    A, B, C = gen.dominant_blocks(N, M, seed=N + M)
    F = gen.uniform_rhs(N, M, K, seed=K)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        assert fac.stencil == 0
        X, info = fac.solve(_t(F), precision=prec, tol=1e-12, return_info=True)
    X = X.cpu().numpy()
    assert info["converged"] and info["rel_res"] <= 1e-12
    assert oracle.rel_res(A, B, C, X, F) <= 2e-12
    assert oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-10
    assert oracle.col_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-10


@pytest.mark.parametrize("prec", PRECISIONS)
def test_refined_poisson_stencil(bt, prec):
    N, M, K, S = 64, 32, 6, 8
    A, B, C = gen.poisson_system(N, M)
    X_exact, F = gen.poisson_manufactured(N, M, K, seed=11)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        assert fac.stencil == 1
        X, info = fac.solve(_t(F), precision=prec, tol=1e-12, return_info=True)
    X = X.cpu().numpy()
    assert info["converged"]
    assert oracle.rel_res(A, B, C, X, F) <= 2e-12
    assert oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-10
    assert oracle.col_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-10


@pytest.mark.parametrize("prec", PRECISIONS)
def test_refined_acoustic_full_size(bt, prec):
    w = gen.config2()
    cols = [0, 130, 300, 511]  # one column in each 128-column tile
    with bt.factor(_t(w.A), _t(w.B), _t(w.C), w.S) as fac:
        X, info = fac.solve(_t(w.F), precision=prec, tol=1e-12, return_info=True)
        X = X.cpu().numpy()
    assert info["converged"] and info["rel_res"] <= 1e-12
    Xr = oracle.solve_block_thomas(w.A, w.B, w.C, w.F[:, :, cols])
    assert oracle.rel_err(X[:, :, cols], Xr) <= 1e-10
    assert oracle.col_err(X[:, :, cols], Xr) <= 1e-10
    assert oracle.rel_res(w.A, w.B, w.C, X[:, :, cols], w.F[:, :, cols]) <= 1e-11


def test_nonconvergence_is_reported(bt):
    A, B, C = gen.dominant_blocks(32, 4, seed=2)
    F = gen.uniform_rhs(32, 4, 3, seed=3)
    with bt.factor(_t(A), _t(B), _t(C), 4) as fac:
        with pytest.raises(bt.BtError) as ei:
            fac.solve(_t(F), precision="f32", tol=1e-300, max_it=1, return_info=True)
        assert ei.value.name == "BT_ERR_NOCONV"


def test_refined_zero_rhs(bt):
    A, B, C = gen.dominant_blocks(16, 3, seed=2)
    with bt.factor(_t(A), _t(B), _t(C), 4) as fac:
        X = fac.solve(torch.zeros((16, 3, 2), dtype=torch.float64, device=DEV), precision="f32")
    assert float(X.abs().max()) == 0.0


# ---------------------------------------------------------------------------
# tensor-core inner solve (tcgen05, BF16 / TF32 operands, FP32 accumulation)
# ---------------------------------------------------------------------------
TC = ["bf16", "tf32", "bf16x3"]


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("N,M,K,S", [
    (64, 64, 20, 8),     # one column tile, ragged
    (48, 128, 70, 6),    # M = 128, one ragged column tile
    (24, 128, 300, 3),   # M = 128, three 128-column tiles, the last ragged
    (40, 64, 130, 20),   # L = 2: one interior row per segment
    (32, 128, 33, 32),   # S = N: every row an interface (no sweep)
    (96, 64, 1, 1),      # S = 1, single right-hand side
])
def test_tc_refined_dense(bt, prec, N, M, K, S):
    A, B, C = gen.dominant_blocks(N, M, seed=N + M + K)
    F = gen.uniform_rhs(N, M, K, seed=K + 1)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        X, info = fac.solve(_t(F), precision=prec, tol=1e-12, return_info=True)
    X = X.cpu().numpy()
    assert info["converged"] and info["rel_res"] <= 1e-12
    assert oracle.rel_res(A, B, C, X, F) <= 2e-12
    assert oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-10
    assert oracle.col_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-10


@pytest.mark.parametrize("prec", TC)
def test_tc_refined_stencil(bt, prec):
    N, M, K, S = 64, 128, 40, 8
    A, B, C = gen.acoustic_system(N, M)
    F = gen.acoustic_rhs(N, M, K, seed=5)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        assert fac.stencil == 1
        X, info = fac.solve(_t(F), precision=prec, tol=1e-12, return_info=True)
    X = X.cpu().numpy()
    assert info["converged"]
    assert oracle.rel_res(A, B, C, X, F) <= 2e-12
    assert oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-10
    assert oracle.col_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-10


@pytest.mark.parametrize("prec", TC)
def test_tc_refined_acoustic_full_size(bt, prec):
    w = gen.config2()
    cols = [0, 130, 300, 511]  # one column in each 128-column tile
    with bt.factor(_t(w.A), _t(w.B), _t(w.C), w.S) as fac:
        X, info = fac.solve(_t(w.F), precision=prec, tol=1e-12, return_info=True)
        X = X.cpu().numpy()
    assert info["converged"] and info["rel_res"] <= 1e-12, info
    Xr = oracle.solve_block_thomas(w.A, w.B, w.C, w.F[:, :, cols])
    assert oracle.rel_err(X[:, :, cols], Xr) <= 1e-10
    assert oracle.col_err(X[:, :, cols], Xr) <= 1e-10


def test_tc_unsupported_block_size(bt):
    # past the largest tile (M > 128) the tensor-core precisions refuse
    A, B, C = gen.dominant_blocks(8, 150, seed=1)
    F = gen.uniform_rhs(8, 150, 2, seed=2)
    with bt.factor(_t(A), _t(B), _t(C), 4) as fac:
        for prec in TC:
            with pytest.raises(bt.BtError) as ei:
                fac.solve(_t(F), precision=prec)
            assert ei.value.name == "BT_ERR_UNSUPPORTED"


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("kind,N,M,K,S", [
    ("dense", 64, 60, 40, 8),       # the paper's block size 60, padded to the 64 tile
    ("dense", 48, 100, 130, 6),     # padded to 128, a ragged 128-column tile
    ("dense", 32, 8, 3, 4),         # a small block
    ("stencil", 64, 30, 33, 8),     # a unit stencil padded to 64 (FP64 stencil residual)
    ("stencil", 40, 120, 20, 5),    # padded to 128
])
def test_tc_refined_padded_block_sizes(bt, prec, kind, N, M, K, S):
    # block sizes below the tiles run on the tensor cores with the factor
    # blocks, interface blocks and panels padded by zero rows and columns
    if kind == "dense":
        A, B, C = gen.dominant_blocks(N, M, seed=N + M)
        F = gen.uniform_rhs(N, M, K, seed=K)
    else:
        A, B, C = gen.acoustic_system(N, M)
        F = gen.acoustic_rhs(N, M, K, seed=K)
    Xr = oracle.solve_block_thomas(A, B, C, F)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        X, info = fac.solve(_t(F), precision=prec, tol=1e-12, return_info=True)
        X0, info0 = fac.solve(_t(F), precision=prec, tol=1.0, return_info=True)
    X = X.cpu().numpy()
    assert info["converged"]
    assert oracle.rel_res(A, B, C, X, F) <= 2e-12
    assert oracle.rel_err(X, Xr) <= 1e-10
    assert oracle.col_err(X, Xr) <= 1e-10
    # the first (unrefined) solve carries the tensor-core precision: it is a solve, not noise
    assert info0["iters"] == 0 and oracle.rel_err(X0.cpu().numpy(), Xr) <= 5e-2


def test_split_precision_needs_fewer_passes(bt):
    # Two-term BF16 operands carry ~2^-17 relative precision: the first solve is
    # far more accurate and refinement needs fewer passes than plain BF16.
    N, M, K, S = 64, 128, 64, 8
    A, B, C = gen.acoustic_system(N, M)
    F = gen.acoustic_rhs(N, M, K, seed=9)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        _, i1 = fac.solve(_t(F), precision="bf16", tol=1e-12, return_info=True)
        X3, i3 = fac.solve(_t(F), precision="bf16x3", tol=1e-12, return_info=True)
    assert i3["rel_res0"] < 1e-2 * i1["rel_res0"], (i1, i3)
    assert i3["iters"] < i1["iters"], (i1, i3)
    assert oracle.rel_err(X3.cpu().numpy(), oracle.solve_block_thomas(A, B, C, F)) <= 1e-10
    assert oracle.col_err(X3.cpu().numpy(), oracle.solve_block_thomas(A, B, C, F)) <= 1e-10


def test_repeated_solves_replay_a_graph(bt):
    # the second call with the same arguments captures the refinement into a
    # CUDA graph, later calls replay it: identical results, and new values in
    # the same F buffer are solved
    N, M, K, S = 64, 128, 96, 8
    A, B, C = gen.acoustic_system(N, M)
    F1 = gen.acoustic_rhs(N, M, K, seed=21)
    F2 = gen.acoustic_rhs(N, M, K, seed=22)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        Fd = _t(F1)
        X = torch.empty_like(Fd)
        X1 = fac.solve(Fd, precision="bf16x3", tol=1e-10, out=X).clone()
        fac.solve(Fd, precision="bf16x3", tol=1e-10, out=X)
        X3 = fac.solve(Fd, precision="bf16x3", tol=1e-10, out=X).clone()
        assert torch.equal(X1, X3)
        Fd.copy_(_t(F2))
        X4, info = fac.solve(Fd, precision="bf16x3", tol=1e-10, out=X, return_info=True)
        assert info["converged"]
        assert oracle.rel_res(A, B, C, X4.cpu().numpy(), F2) <= 1e-10


def test_graph_cache_follows_argument_changes(bt):
    # alternating panel widths and tolerances: every call must solve its own
    # arguments whether it runs directly, captures or replays a graph
    N, M, S = 32, 64, 4
    A, B, C = gen.acoustic_system(N, M)
    Fa = gen.acoustic_rhs(N, M, 96, seed=31)
    Fb = gen.acoustic_rhs(N, M, 40, seed=32)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        Fa_d, Fb_d = _t(Fa), _t(Fb)
        Xa, Xb = torch.empty_like(Fa_d), torch.empty_like(Fb_d)
        for tol, F, Fd, X in [(1e-10, Fa, Fa_d, Xa), (1e-10, Fa, Fa_d, Xa), (1e-10, Fa, Fa_d, Xa),
                              (1e-12, Fb, Fb_d, Xb), (1e-10, Fa, Fa_d, Xa), (1e-12, Fb, Fb_d, Xb),
                              (1e-12, Fb, Fb_d, Xb), (1e-12, Fb, Fb_d, Xb)]:
            _, info = fac.solve(Fd, precision="bf16x3", tol=tol, out=X, return_info=True)
            assert info["converged"] and info["rel_res"] <= tol
            assert oracle.rel_res(A, B, C, X.cpu().numpy(), F) <= 2 * tol


def test_refined_sets_on_concurrent_streams(bt):
    # sets of two factorizations: each factorization's sets in order on its own
    # stream, the two concurrently; three rounds (direct, capture, replay) with
    # new values in one set's F before the last round
    N, M = 64, 64
    mats = [gen.dominant_blocks(N, M, seed=s) for s in (41, 42)]
    Ks = [3, 130, 17, 64, 1]
    Fs_np = [gen.uniform_rhs(N, M, k, seed=60 + i) for i, k in enumerate(Ks)]
    with bt.factor(*(_t(a) for a in mats[0]), 8) as f0, bt.factor(*(_t(a) for a in mats[1]), 16) as f1:
        facs = [f0, f1, f0, f1, f0]
        Fs = [_t(F) for F in Fs_np]
        Xs = [torch.empty_like(F) for F in Fs]
        for rnd in range(3):
            if rnd == 2:
                Fs_np[1] = gen.uniform_rhs(N, M, Ks[1], seed=99)
                Fs[1].copy_(_t(Fs_np[1]))
            bt.solve_refined_sets(facs, Fs, Xs, precision="bf16x3", tol=1e-11)
            torch.cuda.synchronize()
            for i, X in enumerate(Xs):
                A, B, C = mats[i % 2]
                Xr = oracle.solve_block_thomas(A, B, C, Fs_np[i])
                assert oracle.rel_err(X.cpu().numpy(), Xr) <= 1e-10, (rnd, i)
                assert oracle.col_err(X.cpu().numpy(), Xr) <= 1e-10, (rnd, i)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffers_in_overlapped_chunks(bt, pinned):
    # bt_solve_host: K = 300 host columns in chunks of 128, 128 and 44 whose
    # uploads, solves and downloads overlap; FP64 and refined, three calls each
    # (the device panel pairs replay their CUDA graphs from the third)
    N, M, K, S = 64, 64, 300, 8
    A, B, C = gen.dominant_blocks(N, M, seed=51)
    F = gen.uniform_rhs(N, M, K, seed=52)
    Xr = oracle.solve_block_thomas(A, B, C, F)
    Fh = torch.from_numpy(F)
    if pinned:
        Fh = Fh.pin_memory()
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        for prec, bar in (("f64", 1e-12), ("bf16x3", 1e-10)):
            for _ in range(3):
                X = fac.solve(Fh, precision=prec, tol=1e-11)
                assert X.device.type == "cpu" and X.shape == F.shape
                assert oracle.rel_err(X.numpy(), Xr) <= bar, prec
                assert oracle.col_err(X.numpy(), Xr) <= bar, prec


def test_graph_cache_evicts_beyond_its_capacity(bt):
    # 70 argument keys on one handle (more than the 64 graphs a handle keeps),
    # each solved twice (the second call captures): the least recently used
    # graphs are dropped and every solve still returns its own solution
    N, M, S, K = 16, 64, 4, 3
    A, B, C = gen.dominant_blocks(N, M, seed=61)
    F = gen.uniform_rhs(N, M, K, seed=62)
    Xr = oracle.solve_block_thomas(A, B, C, F)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        Fd = _t(F)
        outs = [torch.empty_like(Fd) for _ in range(70)]
        for rnd in range(2):
            for X in outs:
                X.zero_()
                fac.solve(Fd, precision="bf16x3", tol=1e-11, out=X)
        fac.solve(Fd, precision="bf16x3", tol=1e-11, out=outs[0])  # evicted key: runs directly again
        torch.cuda.synchronize()
        for X in outs:
            assert oracle.rel_err(X.cpu().numpy(), Xr) <= 1e-10
            assert oracle.col_err(X.cpu().numpy(), Xr) <= 1e-10


@pytest.mark.parametrize("N,K,S", [
    (64, 40, 8),     # several segments, one ragged column tile
    (32, 130, 16),   # L = 2: one interior row per segment; two column tiles, the last ragged
    (48, 5, 1),      # one segment: no right interface
    (96, 300, 4),    # three column tiles
])
def test_tc_refined_unit_stencil_forward_backward(bt, N, K, S):
    # unit stencil with split BF16 and M = 128: the forward pass accumulating
    # W at each segment's first interior row, step 2.2, and the backward pass
    # forming X from the interface values (no correction kernel)
    M = 128
    A, B, C = gen.acoustic_system(N, M)
    F = gen.acoustic_rhs(N, M, K, seed=N + K)
    Xr = oracle.solve_block_thomas(A, B, C, F)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        assert fac.stencil == 1
        X, info = fac.solve(_t(F), precision="bf16x3", tol=1e-12, return_info=True)
        assert info["converged"], info
        # the first solve alone (no refinement) carries the split-BF16 solve's accuracy
        X0, info0 = fac.solve(_t(F), precision="bf16x3", tol=1.0, return_info=True)
    X = X.cpu().numpy()
    assert oracle.rel_res(A, B, C, X, F) <= 2e-12
    assert oracle.rel_err(X, Xr) <= 1e-10
    assert oracle.col_err(X, Xr) <= 1e-10
    assert info0["iters"] == 0 and info0["rel_res0"] <= 1e-4
    assert oracle.rel_err(X0.cpu().numpy(), Xr) <= 1e-3
