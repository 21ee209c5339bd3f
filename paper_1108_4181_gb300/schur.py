"""Schur-complement CG with a probing band preconditioner (Section 3.3): ctypes
marshalling of the bt_schur_* entry points of libbt.so; every step runs in the
library's CUDA kernels."""

from __future__ import annotations

import ctypes
from typing import Optional

import torch

from . import _lib
from .solver import _as_device_f64, _ptr, _stream_ptr


class SchurPCG:
    """The five-point operator on an nz x nr grid cut by p - 1 interface rows
    into p strips of h rows (nz = p h + p - 1), solved by preconditioned CG on
    the interface Schur complement; strips by the dichotomy (S segments), the
    probing band preconditioner of half-bandwidth d (-1: none) by bt_factor_band."""

    def __init__(self, nr: int, h: int, p: int, shift: float = 0.0, d: int = 2, S: int = 1,
                 device="cuda:0", stream: Optional[torch.cuda.Stream] = None):
        self.device = torch.device(device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = _lib.load().bt_schur_create(int(nr), int(h), int(p), float(shift), int(d), int(S),
                                             _stream_ptr(stream, self.device), ctypes.byref(self._h))
        _lib.check(st, "bt_schur_create")
        q = (ctypes.c_int64 * 8)()
        _lib.check(_lib.load().bt_schur_query(self._h, q), "bt_schur_query")
        self.nr, self.h, self.p, self.nz, self.ng, self.d, self.band_M, self.band_S = (int(v) for v in q)

    def close(self):
        if self._h is not None and self._h.value:
            _lib.load().bt_schur_destroy(self._h)
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

    def _check(self, t: torch.Tensor, rows: int, name: str) -> torch.Tensor:
        t = _as_device_f64(t, self.device, name)
        if t.dim() != 3 or t.shape[0] != rows or t.shape[1] != self.nr:
            raise ValueError(f"{name} must be [{rows}, {self.nr}, K], got {tuple(t.shape)}")
        return t

    def apply(self, v: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        """S v for an interface panel v [p - 1, nr, K]."""
        v = self._check(v, self.p - 1, "v")
        out = torch.empty_like(v)
        _lib.check(_lib.load().bt_schur_apply(self._h, _ptr(v), v.shape[2], _ptr(out),
                                              _stream_ptr(stream, self.device)), "bt_schur_apply")
        return out

    def rhs(self, F: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        """g = f_G - sum_i A_Gi A_ii^{-1} f_i for a grid panel F [nz, nr, K]."""
        F = self._check(F, self.nz, "F")
        g = torch.empty((self.p - 1, self.nr, F.shape[2]), dtype=torch.float64, device=self.device)
        _lib.check(_lib.load().bt_schur_rhs(self._h, _ptr(F), F.shape[2], _ptr(g),
                                            _stream_ptr(stream, self.device)), "bt_schur_rhs")
        return g

    def band(self) -> torch.Tensor:
        """The probing preconditioner in band storage [2d + 1, ng]."""
        if self.d < 0:
            raise ValueError("this solver has no preconditioner (d = -1)")
        ab = torch.empty((2 * self.d + 1, self.ng), dtype=torch.float64, device=self.device)
        torch.cuda.synchronize(self.device)
        _lib.check(_lib.load().bt_schur_band(self._h, _ptr(ab)), "bt_schur_band")
        return ab

    def solve(self, F: torch.Tensor, tol: float = 1e-10, max_it: int = 1000, return_info: bool = False,
              stream: Optional[torch.cuda.Stream] = None, check: bool = True):
        """X [nz, nr, K] with A X = F; info: iterations, converged, rel_res."""
        F = self._check(F, self.nz, "F")
        X = torch.empty_like(F)
        info = _lib.BtInfo()
        st = _lib.load().bt_schur_solve(self._h, _ptr(F), F.shape[2], _ptr(X), float(tol), int(max_it),
                                        _stream_ptr(stream, self.device), ctypes.byref(info))
        if check or st != 4:  # BT_ERR_NOCONV is returned in info when check is False
            _lib.check(st, "bt_schur_solve")
        if return_info:
            return X, dict(iters=info.iters, converged=bool(info.converged), rel_res=info.rel_res)
        return X
