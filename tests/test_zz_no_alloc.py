"""bt_solve_noalloc: the FP64 solve for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc while they run: their device memory belongs
to another allocator (a framework's caching pool or a fixed arena), or they sit
in a latency-bound loop that must not take the device-wide synchronisation that
cudaMalloc and cudaFree may imply.  bt_solve_noalloc serves them with a fixed
scratch array compiled into the library (BT_NOALLOC_SCRATCH_BYTES per device).

This file is collected last on purpose (test_zz_...): if it fails, a run that
stops at the first failure has already run every other test.  It checks, on two
calls in a row with different right-hand sides, that the allocation-free entry
point returns what bt_solve returns (same 1e-12 relative bar as the other FP64
tests), and that a request larger than the fixed array is refused.
"""

import ctypes

import numpy as np
import pytest

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


def test_noalloc_matches_bt_solve_on_two_calls(api):
    bt, _lib, L = api
    N, M, K, S = 64, 16, 9, 8
    A, B, C = gen.dominant_blocks(N, M, seed=7)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    with bt.factor(t(A), t(B), t(C), S) as fac:
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for seed in (11, 12):  # two calls in a row; the second reuses the array left by the first
            F = t(gen.uniform_rhs(N, M, K, seed))
            X_ref = torch.empty_like(F)
            X_na = torch.full_like(F, float("nan"))
            _lib.check(L.bt_solve(fac._h, _p(F), K, _p(X_ref), stream), "bt_solve")
            _lib.check(L.bt_solve_noalloc(fac._h, _p(F), K, _p(X_na), stream), "bt_solve_noalloc")
            torch.cuda.synchronize()
            rel = float(torch.linalg.norm(X_na - X_ref) / torch.linalg.norm(X_ref))
            assert rel <= TOL, rel


def test_noalloc_refuses_requests_beyond_its_array(api):
    bt, _lib, L = api
    N, M, S = 64, 16, 8  # depth 4: scratch = 4 * 8 * 16 * K * 8 bytes
    A, B, C = gen.dominant_blocks(N, M, seed=3)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    K = 4200  # 4.3 MB per column block x 4200 > BT_NOALLOC_SCRATCH_BYTES (16 MiB)
    with bt.factor(t(A), t(B), t(C), S) as fac:
        F = torch.zeros((N, M, K), dtype=torch.float64, device=DEV)
        X = torch.zeros_like(F)
        st = L.bt_solve_noalloc(fac._h, _p(F), K, _p(X), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert _lib.STATUS_NAMES[st] == "BT_ERR_ARG"
        assert b"scratch" in L.bt_last_error()
