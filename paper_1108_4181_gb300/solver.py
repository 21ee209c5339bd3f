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
              stream: Optional[torch.cuda.Stream] = None, residual: str = "auto"):
        """X = P^{-1} F.  F: [N, M, K] float64.

        residual (refined precisions): how F - P X is formed -- "fp64" on the
        CUDA cores, "digits" exactly on the tensor cores (dense blocks, M = 64
        or 128), "auto" the latter where it applies.

        A CUDA tensor is solved in place on the device.  A CPU tensor is the
        end-to-end path (bt_solve_host): its columns go through the device in
        chunks whose uploads, solves and downloads overlap (page-locked F and
        out for the overlap); with return_info the whole panel is copied,
        solved and copied back instead."""
        F = self._panel(F, "F")
        host = F.device.type == "cpu"
        if host and not return_info:
            # columns through the device in overlapped chunks (bt_solve_host)
            if F.dtype != torch.float64:
                raise TypeError("F must be float64")
            Fh = F.contiguous()
            Xh = out if out is not None else torch.empty(F.shape, dtype=torch.float64, pin_memory=F.is_pinned())
            if Xh.device.type != "cpu" or Xh.dtype != torch.float64 or not Xh.is_contiguous() or Xh.shape != F.shape:
                raise ValueError("out must be a contiguous float64 CPU tensor of F's shape")
            opts = _lib.BtOpts(precision=_lib.PREC[precision], max_it=int(max_it), tol=float(tol),
                               stream=_stream_ptr(stream, self.device), k_tile=int(k_tile),
                               residual=_lib.RESIDUAL[residual])
            st = _lib.load().bt_solve_host(self._h, _ptr(Fh), Fh.shape[2], _ptr(Xh), ctypes.byref(opts))
            _lib.check(st, "bt_solve_host")
            return Xh
        if host:
            if F.dtype != torch.float64:
                raise TypeError("F must be float64")
            Fd = F.to(self.device, non_blocking=F.is_pinned())
        else:
            Fd = _as_device_f64(F, self.device, "F")
        K = Fd.shape[2]
        X = out if (out is not None and not host) else torch.empty_like(Fd)
        opts = _lib.BtOpts(precision=_lib.PREC[precision], max_it=int(max_it), tol=float(tol),
                           stream=_stream_ptr(stream, self.device), k_tile=int(k_tile),
                           residual=_lib.RESIDUAL[residual])
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

    def residual(self, F: torch.Tensor, X: torch.Tensor, method: str = "auto",
                 stream: Optional[torch.cuda.Stream] = None):
        """(R, ||R||_F^2) with R = F - P X ([N, M, K] float64, on the device).

        method: "fp64" (CUDA cores), "digits" (exact digit products on the
        tensor cores; dense blocks, M = 64 or 128), "dw" (FP32 double-word
        arithmetic; A_j = B_j = I, C_j = tridiag(-1, c, -1), M % 8 == 0),
        "auto"."""
        F = _as_device_f64(self._panel(F, "F"), self.device, "F")
        X = _as_device_f64(self._panel(X, "X"), self.device, "X")
        if F.shape != X.shape:
            raise ValueError("F and X must have the same shape")
        R = torch.empty_like(F)
        n2 = ctypes.c_double()
        st = _lib.load().bt_residual(self._h, _ptr(F), _ptr(X), F.shape[2], _ptr(R), _lib.RESIDUAL[method],
                                     ctypes.byref(n2), _stream_ptr(stream, self.device))
        _lib.check(st, "bt_residual")
        return R, n2.value

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

    def band(self) -> dict:
        """Diagonal bands of A_j and B_j found at factorisation (c - r of their
        nonzero entries), which the factor GEMMs contract over, and the order n
        of a band-matrix handle (0 otherwise)."""
        q = (ctypes.c_int64 * 5)()
        _lib.check(_lib.load().bt_handle_band(self._h, q), "bt_handle_band")
        return dict(A=(int(q[0]), int(q[1])), B=(int(q[2]), int(q[3])), n=int(q[4]))

    def export(self, what: str) -> torch.Tensor:
        """FP64 factor arrays: 'U', 'V', 'Y' ([N, M, M]) or 'At', 'Ct', 'Bt' ([S, M, M])."""
        code = {"U": 0, "V": 1, "At": 2, "Ct": 3, "Bt": 4, "Y": 5}[what]
        n = self.N if code in (0, 1, 5) else self.S
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


class BandFactorization(Factorization):
    """A factored band matrix of order n (Section 3.3.1, item c), held as the
    block-tridiagonal system of bt_factor_band."""

    def __init__(self, handle: ctypes.c_void_p, device: torch.device):
        super().__init__(handle, device)
        self.n = self.band()["n"]

    def solve(self, F: torch.Tensor, precision: str = "f64", tol: float = 0.0, max_it: int = 0,
              k_tile: int = 0, out: Optional[torch.Tensor] = None, return_info: bool = False,
              stream: Optional[torch.cuda.Stream] = None, residual: str = "auto"):
        """x = Q^{-1} F for F of shape [n] or [n, K] (float64, on the device)."""
        vec = F.dim() == 1
        Fd = _as_device_f64(F.reshape(-1, 1) if vec else F, self.device, "F")
        if Fd.dim() != 2 or Fd.shape[0] != self.n:
            raise ValueError(f"F must be [n] or [n, K] with n = {self.n}, got {tuple(F.shape)}")
        if out is not None and (out.shape != F.shape or out.dtype != torch.float64 or not out.is_contiguous()
                                or out.device != Fd.device):
            raise ValueError("out must be a contiguous float64 tensor of F's shape on F's device")
        X = out.view(Fd.shape) if out is not None else torch.empty_like(Fd)
        opts = _lib.BtOpts(precision=_lib.PREC[precision], max_it=int(max_it), tol=float(tol),
                           stream=_stream_ptr(stream, self.device), k_tile=int(k_tile),
                           residual=_lib.RESIDUAL[residual])
        info = _lib.BtInfo()
        st = _lib.load().bt_solve_band(self._h, _ptr(Fd), Fd.shape[1], _ptr(X), ctypes.byref(opts),
                                       ctypes.byref(info) if return_info else None)
        _lib.check(st, "bt_solve_band")
        X = X.reshape(-1) if vec else X
        if return_info:
            return X, dict(iters=info.iters, converged=bool(info.converged), rel_res=info.rel_res,
                           rel_res0=info.rel_res0)
        return X


def factor_band(ab: torch.Tensor, kl: int, ku: int, M: int, S: int,
                stream: Optional[torch.cuda.Stream] = None) -> BandFactorization:
    """Factor a band matrix given in diagonal-ordered storage ab [kl + ku + 1, n]
    (ab[ku + i - j, j] = Q[i, j]; the layout of LAPACK's and SciPy's banded
    solvers) as a block-tridiagonal matrix of block size M >= kl, ku with S
    segments (S <= ceil(n / M))."""
    if ab.dim() != 2 or ab.shape[0] != kl + ku + 1:
        raise ValueError(f"ab must be [kl + ku + 1, n] = [{kl + ku + 1}, n], got {tuple(ab.shape)}")
    dev = ab.device
    ab = _as_device_f64(ab, dev, "ab")
    h = ctypes.c_void_p()
    with torch.cuda.device(dev):
        st = _lib.load().bt_factor_band(ab.shape[1], int(kl), int(ku), _ptr(ab), int(M), int(S),
                                        _stream_ptr(stream, dev), ctypes.byref(h))
    _lib.check(st, "bt_factor_band")
    return BandFactorization(h, dev)


def _batch_arrays(facs, Fs, Xs):
    n = len(facs)
    if not (len(Fs) == len(Xs) == n) or n < 1:
        raise ValueError("need one F and one X per factorization, n >= 1")
    H = (ctypes.c_void_p * n)(*[f._h.value for f in facs])
    Fp = (ctypes.c_void_p * n)()
    Xp = (ctypes.c_void_p * n)()
    K = (ctypes.c_int64 * n)()
    for i, (f, F, X) in enumerate(zip(facs, Fs, Xs)):
        F = _as_device_f64(f._panel(F, "F"), f.device, "F")
        X = f._panel(X, "X")
        if X.dtype != torch.float64 or X.device != f.device or not X.is_contiguous() or X.shape != F.shape:
            raise ValueError("X must be a contiguous float64 CUDA tensor shaped like F")
        Fp[i], Xp[i], K[i] = F.data_ptr(), X.data_ptr(), F.shape[2]
    return H, Fp, K, Xp


class BatchPlan:
    """A planned batch of solves (bt_batch_*): set i solves facs[i] X_i = F_i.

    precision "f64": one persistent launch for all sets.  Any other precision:
    the sets of each factorization are packed into one panel (each scaled by a
    power of two), refined as one solve per factorization until every set
    meets ``tol`` on its own, and unpacked; all of it is one CUDA graph.  The plan records the tensors' device addresses: keep F and X
    alive and in place while it is used.  run() enqueues one graph launch on
    the current stream."""

    def __init__(self, facs, Fs, Xs, k_tile: int = 0, precision: str = "f64", tol: float = 0.0, max_it: int = 0,
                 residual: str = "auto"):
        self.facs, self.Fs, self.Xs = list(facs), list(Fs), list(Xs)  # keep alive
        self.device = self.facs[0].device
        self.precision = precision
        H, Fp, K, Xp = _batch_arrays(self.facs, self.Fs, self.Xs)
        opts = _lib.BtOpts(precision=_lib.PREC[precision], max_it=int(max_it), tol=float(tol), stream=None,
                           k_tile=int(k_tile), residual=_lib.RESIDUAL[residual])
        self._b = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(_lib.load().bt_batch_create(len(self.facs), H, Fp, K, Xp, ctypes.byref(opts),
                                                   ctypes.byref(self._b)), "bt_batch_create")
        q = (ctypes.c_int64 * 6)()
        _lib.check(_lib.load().bt_batch_query(self._b, q), "bt_batch_query")
        self.items, self.stages, self.ctas, self.threads, self.k_tile, self.graph = (int(v) for v in q)

    def info(self, i: int):
        """The refinement report of set i's factorization group (after status())."""
        inf = _lib.BtInfo()
        _lib.check(_lib.load().bt_batch_info(self._b, int(i), ctypes.byref(inf)), "bt_batch_info")
        return dict(iters=inf.iters, converged=bool(inf.converged), rel_res=inf.rel_res, rel_res0=inf.rel_res0)

    def run(self, stream: Optional[torch.cuda.Stream] = None):
        _lib.check(_lib.load().bt_batch_run(self._b, _stream_ptr(stream, self.device)), "bt_batch_run")

    def status(self):
        """Waits for the plan's work; raises if a bounded wait gave up or a
        refined group did not converge."""
        _lib.check(_lib.load().bt_batch_status(self._b), "bt_batch_status")

    def debug(self, limit_s: float = 0.0, skip_stage: int = -1):
        """Diagnostics (bt_batch_debug): the grid-barrier wait limit of later
        runs (0 = default) and a planted failure (CTA 0 leaves instead of
        arriving at the barrier after stage `skip_stage`; -1 = none)."""
        _lib.check(_lib.load().bt_batch_debug(self._b, float(limit_s), int(skip_stage)), "bt_batch_debug")

    def close(self):
        if self._b is not None and self._b.value:
            _lib.load().bt_batch_destroy(self._b)
        self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(facs, Fs, Xs=None, k_tile: int = 0, stream: Optional[torch.cuda.Stream] = None):
    """X_i = P_i^{-1} F_i for every set i in one persistent launch (FP64, bt_solve_batched)."""
    if Xs is None:
        Xs = [torch.empty_like(F) for F in Fs]
    H, Fp, K, Xp = _batch_arrays(facs, Fs, Xs)
    dev = facs[0].device
    opts = _lib.BtOpts(precision=0, max_it=0, tol=0.0, stream=_stream_ptr(stream, dev), k_tile=int(k_tile),
                       residual=0)
    with torch.cuda.device(dev):
        _lib.check(_lib.load().bt_solve_batched(len(facs), H, Fp, K, Xp, ctypes.byref(opts)), "bt_solve_batched")
    return Xs


def solve_refined_sets(facs, Fs, Xs=None, precision: str = "bf16x3", tol: float = 0.0, max_it: int = 0,
                       residual: str = "auto"):
    """Refined solves of many right-hand-side sets, X_b = P_{facs[b]}^{-1} F_b,
    through a refined BatchPlan (one CUDA graph; every set meets ``tol`` on its
    own).  Plans once per call: keep a BatchPlan to run the same sets again.
    The work is ordered on the current stream; returns the outputs."""
    if Xs is None:
        Xs = [torch.empty_like(F) for F in Fs]
    if not (len(facs) == len(Fs) == len(Xs)):
        raise ValueError("facs, Fs and Xs must have the same length")
    if not facs:
        return Xs
    plan = BatchPlan(facs, Fs, Xs, precision=precision, tol=tol, max_it=max_it, residual=residual)
    plan.run()
    plan.status()
    plan.close()
    return Xs
    dev = Fs[0].device
    cur = torch.cuda.current_stream(dev)
    used = {}
    for fac, F, X in zip(facs, Fs, Xs):
        st = used.get(id(fac))
        if st is None:
            st = getattr(fac, "_side_stream", None)
            if st is None:
                st = torch.cuda.Stream(dev)
                fac._side_stream = st
            st.wait_stream(cur)  # the inputs are ready on the current stream
            used[id(fac)] = st
        fac.solve(F, precision=precision, tol=tol, max_it=max_it, out=X, stream=st, residual=residual)
    for st in used.values():
        cur.wait_stream(st)
    return Xs
