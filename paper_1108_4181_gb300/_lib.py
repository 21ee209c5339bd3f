"""ctypes binding of libbt.so: argument marshalling only.

Every arithmetic step runs inside the library's CUDA kernels.  If the library
is missing or cannot be loaded, the calls below raise; nothing falls back to
the CPU.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbt.so")

BT_OK = 0
STATUS_NAMES = {
    0: "BT_OK", 1: "BT_ERR_ARG", 2: "BT_ERR_SINGULAR", 3: "BT_ERR_CUDA", 4: "BT_ERR_NOCONV",
    5: "BT_ERR_TIMEOUT", 6: "BT_ERR_OOM", 7: "BT_ERR_UNSUPPORTED",
}
# bytes of the fixed scratch array of bt_solve_noalloc (BT_NOALLOC_SCRATCH_BYTES in bt.h)
NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024
PREC = {"f64": 0, "tf32": 1, "bf16": 2, "f32": 3, "bf16x3": 4}
RESIDUAL = {"auto": 0, "fp64": 1, "digits": 2, "dw": 3}

# Every symbol declared in include/bt.h, with (restype, argtypes).
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


class BtOpts(ctypes.Structure):
    _fields_ = [("precision", _i32), ("max_it", _i32), ("tol", ctypes.c_double), ("stream", _vp),
                ("k_tile", _i32), ("residual", _i32)]


class BtInfo(ctypes.Structure):
    _fields_ = [("iters", _i32), ("converged", _i32), ("rel_res", ctypes.c_double),
                ("rel_res0", ctypes.c_double)]


class BtKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", _i64), ("total_ms", ctypes.c_double)]


SIGNATURES = {
    "bt_factor": (ctypes.c_int, [_i64, _i64, _vp, _vp, _vp, _i64, _vp, ctypes.POINTER(_vp)]),
    "bt_solve": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "bt_solve_ex": (ctypes.c_int, [_vp, _vp, _i64, _vp, ctypes.POINTER(BtOpts), ctypes.POINTER(BtInfo)]),
    "bt_solve_host": (ctypes.c_int, [_vp, _vp, _i64, _vp, ctypes.POINTER(BtOpts)]),
    "bt_factor_band": (ctypes.c_int, [_i64, _i64, _i64, _vp, _i64, _i64, _vp, ctypes.POINTER(_vp)]),
    "bt_solve_band": (ctypes.c_int, [_vp, _vp, _i64, _vp, ctypes.POINTER(BtOpts), ctypes.POINTER(BtInfo)]),
    "bt_handle_band": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "bt_schur_create": (ctypes.c_int, [_i64, _i64, _i64, ctypes.c_double, _i64, _i64, _vp, ctypes.POINTER(_vp)]),
    "bt_schur_apply": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "bt_schur_rhs": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "bt_schur_solve": (ctypes.c_int, [_vp, _vp, _i64, _vp, ctypes.c_double, _i32, _vp, ctypes.POINTER(BtInfo)]),
    "bt_schur_band": (ctypes.c_int, [_vp, _vp]),
    "bt_schur_query": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "bt_schur_destroy": (None, [_vp]),
    "bt_solve_adjoint": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    "bt_residual": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _i32, ctypes.POINTER(ctypes.c_double), _vp]),
    "bt_destroy": (None, [_vp]),
    "bt_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "bt_last_error": (ctypes.c_char_p, []),
    "bt_handle_query": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "bt_factor_export": (ctypes.c_int, [_vp, _i32, _vp]),
    "bt_solve_stages": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i32, _vp]),
    "bt_solve_noalloc": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "bt_profile_enable": (ctypes.c_int, [_vp, _i32]),
    "bt_profile_read": (ctypes.c_int, [_vp, ctypes.POINTER(BtKernelStat), _i32, ctypes.POINTER(_i32)]),
    "bt_batch_create": (ctypes.c_int, [_i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_i64),
                                       ctypes.POINTER(_vp), ctypes.POINTER(BtOpts), ctypes.POINTER(_vp)]),
    "bt_batch_run": (ctypes.c_int, [_vp, _vp]),
    "bt_batch_status": (ctypes.c_int, [_vp]),
    "bt_batch_query": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "bt_batch_info": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(BtInfo)]),
    "bt_batch_debug": (ctypes.c_int, [_vp, ctypes.c_double, _i32]),
    "bt_batch_destroy": (None, [_vp]),
    "bt_solve_batched": (ctypes.c_int, [_i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_i64),
                                        ctypes.POINTER(_vp), ctypes.POINTER(BtOpts)]),
}

_LIB = None


class BtError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


def load(path: str = LIB_PATH):
    """Load libbt.so (built in-tree by build.py) and declare its signatures."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it first (python -m paper_1108_4181_gb300.build)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(status: int, where: str):
    if status != BT_OK:
        lib = load()
        detail = lib.bt_last_error().decode(errors="replace")
        raise BtError(status, where, detail)
