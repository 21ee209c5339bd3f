"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point that include/bt.h declares (no compute calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "bt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bt_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1108_4181_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ("bt_factor", "bt_solve", "bt_solve_ex", "bt_solve_adjoint", "bt_destroy", "bt_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, f"declared in bt.h but not exported: {missing}"


def test_binding_signatures_cover_the_header():
    from paper_1108_4181_gb300 import _lib

    assert sorted(_lib.SIGNATURES) == _declared_symbols()


def test_strerror_and_argument_errors_without_gpu(lib):
    from paper_1108_4181_gb300 import _lib

    L = _lib.load()
    assert L.bt_strerror(0) == b"ok"
    assert L.bt_strerror(2).startswith(b"singular")
    h = ctypes.c_void_p()
    # N % S != 0 is rejected on the host before any device call.
    st = L.bt_factor(10, 2, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), 3, None, ctypes.byref(h))
    assert st == 1
    assert b"N % S" in L.bt_last_error()
    # NULL handle / K = 0 rejected
    assert L.bt_solve(None, ctypes.c_void_p(8), 1, ctypes.c_void_p(16), None) == 1
    assert L.bt_solve_stages(None, ctypes.c_void_p(8), 0, ctypes.c_void_p(16), 3, None) == 1


def test_band_argument_errors_without_gpu(lib):
    from paper_1108_4181_gb300 import _lib

    L = _lib.load()
    h = ctypes.c_void_p()
    p = ctypes.c_void_p(8)
    # kl > M, ku > M, S > ceil(n / M), n = 0, NULL storage: rejected on the host
    for args in [(100, 9, 3, p, 8, 1), (100, 3, 9, p, 8, 1), (100, 3, 3, p, 8, 14), (0, 1, 1, p, 8, 1),
                 (100, 3, 3, None, 8, 1)]:
        assert L.bt_factor_band(*args, None, ctypes.byref(h)) == 1
        assert not h.value
    assert L.bt_solve_band(None, p, 1, ctypes.c_void_p(16), None, None) == 1
    out = (ctypes.c_int64 * 5)()
    assert L.bt_handle_band(None, out) == 1


def test_schur_argument_errors_without_gpu(lib):
    from paper_1108_4181_gb300 import _lib

    L = _lib.load()
    h = ctypes.c_void_p()
    # p < 2, nr % S != 0, d >= ng, negative shift, h > 1024: rejected on the host
    for args in [(16, 4, 1, 0.0, 1, 1), (16, 4, 2, 0.0, 1, 3), (16, 4, 2, 0.0, 16, 1), (16, 4, 2, -1.0, 1, 1),
                 (16, 1025, 2, 0.0, 1, 1), (16, 4, 2, 0.0, -2, 1)]:
        assert L.bt_schur_create(*args, None, ctypes.byref(h)) == 1
        assert not h.value
    assert L.bt_schur_solve(None, ctypes.c_void_p(8), 1, ctypes.c_void_p(16), 1e-8, 10, None, None) == 1
    assert L.bt_schur_apply(None, ctypes.c_void_p(8), 1, ctypes.c_void_p(16), None) == 1


def test_noalloc_scratch_size_matches_the_header():
    from paper_1108_4181_gb300 import _lib

    src = open(os.path.join(ROOT, "include", "bt.h")).read()
    m = re.search(r"#define\s+BT_NOALLOC_SCRATCH_BYTES\s+\((\d+)u\s*\*\s*(\d+)u\s*\*\s*(\d+)u\)", src)
    assert m, "BT_NOALLOC_SCRATCH_BYTES not found in bt.h"
    assert _lib.NOALLOC_SCRATCH_BYTES == int(m.group(1)) * int(m.group(2)) * int(m.group(3))
