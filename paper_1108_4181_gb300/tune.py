"""Autotuner for the segment count S and the right-hand-side tile.

S trades the length of the sequential segment sweeps (L = N/S rows) against
the size of the reduced system and its dichotomy tree (S interfaces, depth
ceil(log2(S+1))); the tile sets how many right-hand-side columns one CTA (or
one work item of a batch) carries.  The tuner factors the matrices once per
candidate S, times the candidate launches on the device with CUDA events, and
keeps the fastest.  Timing and bookkeeping only: every solve it times runs in
the library's kernels.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import solver

S_CANDIDATES = (32, 64, 128, 256)


@dataclass
class TuneResult:
    S: int
    k_tile: int
    ms: float
    table: Dict[Tuple[int, int], float] = field(default_factory=dict)  # (S, k_tile) -> ms per run
    factors: Optional[List[solver.Factorization]] = None  # the winner's factorizations (kept open)
    plan: Optional["solver.BatchPlan"] = None  # tune_batched_refined: the winner's plan (kept open)


def _valid_S(N: int, cands: Sequence[int]) -> List[int]:
    out = [s for s in cands if 1 <= s <= N and N % s == 0]
    if not out:
        raise ValueError(f"no candidate S divides N = {N}")
    return out


def _time(fn, reps: int, device) -> float:
    fn()  # warm-up (first-use allocations, graph instantiation)
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(device)
    best = float("inf")
    for _ in range(reps):
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_batched(mats, sets, S_candidates: Sequence[int] = S_CANDIDATES,
                 tiles: Sequence[int] = (0, 4, 8, 16), reps: int = 3) -> TuneResult:
    """Best (S, k_tile) for a batch.

    mats: list of (A, B, C) float64 CUDA tensors [N, M, M]; sets: list of
    (matrix index, F [N, M, K] float64 CUDA tensor).  Returns the winner with
    its factorizations kept open (``result.factors``)."""
    N = mats[0][0].shape[0]
    device = mats[0][0].device
    Fs = [F for _, F in sets]
    Xs = [torch.empty_like(F) for F in Fs]
    table: Dict[Tuple[int, int], float] = {}
    best: Optional[TuneResult] = None
    for S in _valid_S(N, S_candidates):
        facs = [solver.factor(A, B, C, S) for A, B, C in mats]
        keep = False
        for kt in tiles:
            plan = solver.BatchPlan([facs[i] for i, _ in sets], Fs, Xs, k_tile=kt)
            ms = _time(plan.run, reps, device)
            plan.status()
            plan.close()
            table[(S, plan.k_tile)] = ms
            if best is None or ms < best.ms:
                if best is not None and best.factors is not None and best.factors is not facs:
                    for f in best.factors:
                        f.close()
                best = TuneResult(S=S, k_tile=plan.k_tile, ms=ms, factors=facs)
                keep = True
        if not keep:
            for f in facs:
                f.close()
    best.table = table
    return best


def tune_batched_refined(mats, sets, precision: str = "bf16x3", tol: float = 0.0,
                         S_candidates: Sequence[int] = (32, 64, 128), reps: int = 2) -> TuneResult:
    """Best S for the refined (mixed-precision) batch: for each candidate, every
    matrix is factored and a refined ``solver.BatchPlan`` (the sets of a matrix
    packed into one panel, one CUDA graph) is timed.  Same arguments and result
    as ``tune_batched`` (k_tile 0: the tensor-core tile); the winner's plan is
    kept in ``result.plan``."""
    N = mats[0][0].shape[0]
    device = mats[0][0].device
    Xs = [torch.empty_like(F) for _, F in sets]
    table: Dict[Tuple[int, int], float] = {}
    best: Optional[TuneResult] = None
    best_plan = None
    for S in _valid_S(N, S_candidates):
        facs = [solver.factor(A, B, C, S) for A, B, C in mats]
        plan = solver.BatchPlan([facs[i] for i, _ in sets], [F for _, F in sets], Xs, precision=precision, tol=tol)

        def step():
            plan.run()

        step()
        plan.status()
        ms = _time(step, reps, device)
        plan.status()
        table[(S, 0)] = ms
        if best is None or ms < best.ms:
            if best is not None:
                best_plan.close()
                for f in best.factors:
                    f.close()
            best = TuneResult(S=S, k_tile=0, ms=ms, factors=facs)
            best_plan = plan
        else:
            plan.close()
            for f in facs:
                f.close()
    best.table = table
    best.plan = best_plan
    return best


def tune_solve(A, B, C, F, precision: str = "f64", tol: float = 0.0,
               S_candidates: Sequence[int] = S_CANDIDATES, reps: int = 3) -> TuneResult:
    """Best S for repeated solves of F-shaped panels against one matrix."""
    N = A.shape[0]
    X = torch.empty_like(F)
    table: Dict[Tuple[int, int], float] = {}
    best: Optional[TuneResult] = None
    for S in _valid_S(N, S_candidates):
        fac = solver.factor(A, B, C, S)
        ms = _time(lambda: fac.solve(F, precision=precision, tol=tol, out=X), reps, F.device)
        table[(S, 0)] = ms
        if best is None or ms < best.ms:
            if best is not None:
                best.factors[0].close()
            best = TuneResult(S=S, k_tile=0, ms=ms, factors=[fac])
        else:
            fac.close()
    best.table = table
    return best
