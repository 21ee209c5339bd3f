"""Python face of the C ABI: device memory and streams come from PyTorch, every
arithmetic step runs in libbt's CUDA kernels (argument marshalling only here)."""

from __future__ import annotations

import ctypes
from typing import Optional

import torch

from . import _lib


def _stream_ptr(stream: Optional[torch.cuda.Stream], device) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _as_device_f64(t: torch.Tensor, device, name: str) -> torch.Tensor:
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64, got {t.dtype}")
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, the factorisation on {device}")
    return t.contiguous()


class Factorization:
    """A factored block-tridiagonal matrix (Algorithm 2, stage 1) held on one GPU."""

    def __init__(self, handle: ctypes.c_void_p, device: torch.device):
        self._h = handle
        self.device = device
        q = (ctypes.c_int64 * 6)()
        _lib.check(_lib.load().bt_handle_query(self._h, q), "bt_handle_query")
        self.N, self.M, self.S, self.depth, self.stencil, self.device_bytes = (int(v) for v in q)

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if self._h is not None and self._h.value:
            _lib.load().bt_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- shapes ---------------------------------------------------------------
    def _panel(self, F: torch.Tensor, name: str) -> torch.Tensor:
        if F.dim() == 2:
            F = F.reshape(self.N, self.M, F.shape[1])
        if F.dim() != 3 or F.shape[0] != self.N or F.shape[1] != self.M:
            raise ValueError(f"{name} must be [N, M, K] = [{self.N}, {self.M}, K], got {tuple(F.shape)}")
        return F

    # -- stage 2 -------------------------------------------------------------
    def solve(self, F: torch.Tensor, precision: str = "f64", tol: float = 0.0, max_it: int = 0,
              k_tile: int = 0, out: Optional[torch.Tensor] = None, return_info: bool = False,
              stream: Optional[torch.cuda.Stream] = None):
        """X = P^{-1} F.  F: [N, M, K] float64.

        A CUDA tensor is solved in place on the device.  A CPU tensor is the
        end-to-end path: it is copied to the device (through pinned memory when
        F is pinned), solved, and the result copied back to a CPU tensor."""
        F = self._panel(F, "F")
        host = F.device.type == "cpu"
        if host:
            if F.dtype != torch.float64:
                raise TypeError("F must be float64")
            Fd = F.to(self.device, non_blocking=F.is_pinned())
        else:
            Fd = _as_device_f64(F, self.device, "F")
        K = Fd.shape[2]
        X = out if (out is not None and not host) else torch.empty_like(Fd)
        opts = _lib.BtOpts(precision=_lib.PREC[precision], max_it=int(max_it), tol=float(tol),
                           stream=_stream_ptr(stream, self.device), k_tile=int(k_tile), reserved=0)
        info = _lib.BtInfo()
        st = _lib.load().bt_solve_ex(self._h, _ptr(Fd), K, _ptr(X), ctypes.byref(opts),
                                     ctypes.byref(info) if return_info else None)
        _lib.check(st, "bt_solve_ex")
        if host:
            Xh = out if out is not None else torch.empty(F.shape, dtype=torch.float64, pin_memory=F.is_pinned())
            Xh.copy_(X, non_blocking=False)
            X = Xh
        if return_info:
            return X, dict(iters=info.iters, converged=bool(info.converged), rel_res=info.rel_res,
                           rel_res0=info.rel_res0)
        return X

    def solve_stages(self, F: torch.Tensor, stages: int, X: Optional[torch.Tensor] = None,
                     stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        """Runs the first `stages` steps of the FP64 pipeline (diagnostics)."""
        F = _as_device_f64(self._panel(F, "F"), self.device, "F")
        if X is None:
            X = torch.zeros_like(F)
        st = _lib.load().bt_solve_stages(self._h, _ptr(F), F.shape[2], _ptr(X), int(stages),
                                         _stream_ptr(stream, self.device))
        _lib.check(st, "bt_solve_stages")
        return X

    def export(self, what: str) -> torch.Tensor:
        """FP64 factor arrays: 'U', 'V' ([N, M, M]) or 'At', 'Ct', 'Bt' ([S, M, M])."""
        code = {"U": 0, "V": 1, "At": 2, "Ct": 3, "Bt": 4}[what]
        n = self.N if code < 2 else self.S
        dst = torch.empty((n, self.M, self.M), dtype=torch.float64, device=self.device)
        torch.cuda.synchronize(self.device)
        _lib.check(_lib.load().bt_factor_export(self._h, code, _ptr(dst)), "bt_factor_export")
        return dst

    def profile(self, enable: bool):
        """Turn per-kernel CUDA-event timing of later launches on or off."""
        _lib.check(_lib.load().bt_profile_enable(self._h, 1 if enable else 0), "bt_profile_enable")

    def profile_read(self) -> dict:
        """{kernel name: (launches, total device ms)} since the last read."""
        cap = 64
        buf = (_lib.BtKernelStat * cap)()
        n = ctypes.c_int32()
        _lib.check(_lib.load().bt_profile_read(self._h, buf, cap, ctypes.byref(n)), "bt_profile_read")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n.value, cap))}

    def adjoint(self, X: torch.Tensor, G: torch.Tensor, want=("F", "A", "B", "C"),
                stream: Optional[torch.cuda.Stream] = None):
        """(dF, dA, dB, dC) for upstream gradient G = dL/dX at the solution X."""
        X = _as_device_f64(self._panel(X, "X"), self.device, "X")
        G = _as_device_f64(self._panel(G, "G"), self.device, "G")
        K = X.shape[2]
        dF = torch.empty_like(G) if "F" in want else None
        blk = lambda: torch.empty((self.N, self.M, self.M), dtype=torch.float64, device=self.device)
        dA = blk() if "A" in want else None
        dB = blk() if "B" in want else None
        dC = blk() if "C" in want else None
        st = _lib.load().bt_solve_adjoint(self._h, _ptr(X), _ptr(G), K, _ptr(dF), _ptr(dA), _ptr(dB), _ptr(dC),
                                          _stream_ptr(stream, self.device))
        _lib.check(st, "bt_solve_adjoint")
        return dF, dA, dB, dC


def factor(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, S: int,
           stream: Optional[torch.cuda.Stream] = None) -> Factorization:
    """Factor P (blocks [N, M, M] float64 CUDA tensors) with S segments (N % S == 0)."""
    if A.shape != B.shape or A.shape != C.shape or A.dim() != 3 or A.shape[1] != A.shape[2]:
        raise ValueError("A, B, C must all be [N, M, M]")
    dev = C.device
    A = _as_device_f64(A, dev, "A")
    B = _as_device_f64(B, dev, "B")
    C = _as_device_f64(C, dev, "C")
    N, M = A.shape[0], A.shape[1]
    h = ctypes.c_void_p()
    with torch.cuda.device(dev):
        st = _lib.load().bt_factor(N, M, _ptr(A), _ptr(B), _ptr(C), int(S), _stream_ptr(stream, dev),
                                   ctypes.byref(h))
    _lib.check(st, "bt_factor")
    return Factorization(h, dev)
