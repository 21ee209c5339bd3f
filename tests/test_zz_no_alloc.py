"""bt_solve_noalloc: the FP64 solve for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc while they run: their device memory belongs
to another allocator (a framework's caching pool or a fixed arena), or they sit
in a latency-bound loop that must not take the device-wide synchronisation that
cudaMalloc and cudaFree may imply.  bt_solve_noalloc serves them with a fixed
scratch array compiled into the library (BT_NOALLOC_SCRATCH_BYTES per device).

This file is collected last on purpose (test_zz_...): if it fails, a run that
stops at the first failure has already run every other test.  It checks, on two
calls in a row with different right-hand sides, that the allocation-free entry
point returns what bt_solve returns and what the CPU oracle returns, column by
column (same 1e-12 relative bar as the other FP64 tests), and that the size
limit sits exactly where depth*S*M*K*8 passes the fixed array's size.
"""

import ctypes

import numpy as np
import pytest

import oracle
from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-12


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def api():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1108_4181_gb300 as bt
    from paper_1108_4181_gb300 import _lib

    return bt, _lib, _lib.load()


def _colwise_rel(X, Xr):
    """Largest over columns of max_i |X - Xr| / max_i |Xr| (each column of the
    (N*M) x K panel on its own)."""
    X = X.reshape(-1, X.shape[-1])
    Xr = Xr.reshape(-1, Xr.shape[-1])
    return float(np.max(np.max(np.abs(X - Xr), axis=0) / np.max(np.abs(Xr), axis=0)))


def test_noalloc_matches_bt_solve_on_two_calls(api):
    bt, _lib, L = api
    N, M, K, S = 64, 16, 9, 8
    A, B, C = gen.dominant_blocks(N, M, seed=7)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    with bt.factor(t(A), t(B), t(C), S) as fac:
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for seed in (11, 12):  # two calls in a row; the second reuses the array left by the first
            Fh = gen.uniform_rhs(N, M, K, seed)
            F = t(Fh)
            X_ref = torch.empty_like(F)
            X_na = torch.full_like(F, float("nan"))
            _lib.check(L.bt_solve(fac._h, _p(F), K, _p(X_ref), stream), "bt_solve")
            _lib.check(L.bt_solve_noalloc(fac._h, _p(F), K, _p(X_na), stream), "bt_solve_noalloc")
            torch.cuda.synchronize()
            rel = float(torch.linalg.norm(X_na - X_ref) / torch.linalg.norm(X_ref))
            assert rel <= TOL, rel
            X_or = oracle.solve_block_thomas(A, B, C, Fh)
            X_na_h = X_na.cpu().numpy()
            assert oracle.rel_err(X_na_h, X_or) <= TOL
            assert _colwise_rel(X_na_h, X_or) <= TOL


def test_noalloc_refuses_requests_beyond_its_array(api):
    bt, _lib, L = api
    N, M, S = 64, 16, 8
    A, B, C = gen.dominant_blocks(N, M, seed=3)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    limit = _lib.NOALLOC_SCRATCH_BYTES
    with bt.factor(t(A), t(B), t(C), S) as fac:
        q = (ctypes.c_int64 * 6)()
        _lib.check(L.bt_handle_query(fac._h, q), "bt_handle_query")
        depth = int(q[3])
        per_col = depth * S * M * 8  # scratch bytes per right-hand-side column
        k_max = limit // per_col     # the largest K that fits the array
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        F = torch.zeros((N, M, k_max + 1), dtype=torch.float64, device=DEV)
        X = torch.zeros_like(F)
        st = L.bt_solve_noalloc(fac._h, _p(F), k_max + 1, _p(X), stream)
        assert _lib.STATUS_NAMES[st] == "BT_ERR_ARG"
        assert b"scratch" in L.bt_last_error()
        # a K whose product with depth*S*M*8 wraps 64 bits is refused too
        st = L.bt_solve_noalloc(fac._h, _p(F), (1 << 63) // per_col * 2 + 1, _p(X), stream)
        assert _lib.STATUS_NAMES[st] == "BT_ERR_ARG"
        # the largest K that fits is accepted (a panel with K = k_max columns)
        Fk = F[..., :k_max].contiguous()
        Xk = torch.full_like(Fk, float("nan"))
        _lib.check(L.bt_solve_noalloc(fac._h, _p(Fk), k_max, _p(Xk), stream), "bt_solve_noalloc at the limit")
        torch.cuda.synchronize()
        assert bool(torch.all(Xk == 0.0))  # F = 0 gives X = 0
