"""Benchmark of the block-tridiagonal dichotomy solve (Algorithm 2, stage 2).

Workload: the acoustic-style shifted five-point operator with absorbing-layer
damping, N = 4096 block rows, M = 128, K = 512 right-hand sides, S = 64
segments (synthetic, seeded; the stand-in for the paper's "same matrix, many
right-hand sides" Laguerre-harmonic workload).  One step = one complete solve
of the 512-column panel (every step of stage 2, plus refinement passes in the
mixed precisions) with F already resident in HBM; the factorisation (stage 1,
the paper's "Pre") is done once before timing and reported separately.

Prints one JSON line (rank 0).  `--impl reference` times the CPU FP64 oracle
on a bounded column sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "unknowns solved/s (N*M*K) at rel. error <=1e-10; mixed vs FP64 GPU speedup"
N, M, K, S = 4096, 128, 512, 64
WORKLOAD = f"acoustic PML operator N={N} M={M} K={K} S={S} (tridiag C, A=B=I)"
ORACLE_COLS = 64  # bounded CPU sample: 64 of the 512 right-hand sides
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e-3  # SMs x FP64 FMA/clk/SM x 2 flop x GHz -> TFLOP/s


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload(rank: int):
    from workloads import gen

    # every rank solves its own 512 columns against the same matrix (weak scaling)
    A, B, C = gen.acoustic_system(N, M)
    F = gen.acoustic_rhs(N, M, K, seed=2 + 1000 * rank)
    return A, B, C, F


def _oracle_sample(A, B, C, F_cols):
    import oracle

    t0 = time.perf_counter()
    X = oracle.solve_block_thomas(A, B, C, F_cols)
    return X, time.perf_counter() - t0


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from workloads import gen

    A, B, C = gen.acoustic_system(N, M)
    cols = list(range(ORACLE_COLS))
    Fs = gen.acoustic_rhs(N, M, K, seed=2, columns=cols)
    for _ in range(args.warmup):
        _oracle_sample(A, B, C, Fs[:, :, :8])
    times = []
    for _ in range(args.steps):
        _, t = _oracle_sample(A, B, C, Fs)
        times.append(t)
    t = float(np.mean(times))
    value = N * M * len(cols) / t
    cores = len(os.sched_getaffinity(0))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{len(cols)} of {K} right-hand sides per step"},
        "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 block-sweep oracle (numpy/LAPACK) on {len(cols)} of {K} columns, full N and M"},
        "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1108_4181_gb300 as bt

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hbm_peak, bf16_peak, bf16_sus, peak_kind = _peaks()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    A, B, C, F = _workload(rank)
    At, Bt, Ct = (torch.from_numpy(a).to(dev) for a in (A, B, C))
    F_host = torch.from_numpy(F).pin_memory()
    Fd = F_host.to(dev)
    del F
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    fac = bt.factor(At, Bt, Ct, S)
    torch.cuda.synchronize(dev)
    pre_s = time.perf_counter() - t0
    del At, Bt, Ct

    precision = args.precision
    X = torch.empty_like(Fd)
    stream = torch.cuda.current_stream(dev)

    def step(out):
        return fac.solve(Fd, precision=precision, tol=args.tol, out=out)

    for _ in range(max(3, args.warmup)):
        step(X)
    barrier()
    fac.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step(X)
        e1.record(stream)
        barrier()
    fac.profile(False)
    prof = fac.profile_read()
    ms = e0.elapsed_time(e1)
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    unknowns = N * M * K
    value = unknowns * ws / (ms_step * 1e-3)
    launches = sum(v[0] for v in prof.values())

    # refinement report of one more solve (untimed)
    _, info = fac.solve(Fd, precision=precision, tol=args.tol, out=X, return_info=True)

    # end-to-end: host F (pinned) -> device -> solve -> host X, through the public API
    Xh = torch.empty(F_host.shape, dtype=torch.float64, pin_memory=True)
    for _ in range(1):
        fac.solve(F_host, precision=precision, tol=args.tol, out=Xh)
    barrier()
    e2e_steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        fac.solve(F_host, precision=precision, tol=args.tol, out=Xh)
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if ws > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = unknowns * ws / e2e_s

    # roofline of the dominant kernel
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else ("none", (1, 1.0))
    dom_name, (dom_launches, dom_ms) = dom
    avg_s = dom_ms / max(1, dom_launches) * 1e-3
    L = N // S
    if dom_name == "f64_sweep":
        flops = 2.0 * M * M * K * S * (3 * L - 5)
        roof = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "kernel": dom_name, "peak_kind": "nominal FP64 FMA rate (152 SMs x 2 FMA/clk x 2.07 GHz)"}
    elif dom_name == "f64_correct":
        flops = 2.0 * 2 * M * M * K * (N - S)
        roof = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "kernel": dom_name, "peak_kind": "nominal FP64 FMA rate (152 SMs x 2 FMA/clk x 2.07 GHz)"}
    else:
        roof = {"bound": "unknown", "achieved": None, "peak": None, "unit": None, "kernel": dom_name}
    if roof.get("achieved") is not None:
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["kernels_ms_per_step"] = {k: v[1] / args.steps for k, v in prof.items()}

    line = {
        "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32+f64", "tf32": "tf32+f64", "bf16": "bf16+f64", "bf16x3": "bf16x3+f64"}[precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": precision, "tol": args.tol,
                   "l2": "inputs larger than L2 (F, X 2.1 GB each)", "pre_s": pre_s,
                   "parallelism": f"K-replicas x{ws}" if ws > 1 else "single GPU"},
        "gpu_launches": launches,
        "refinement": info,
        "e2e": {"value": e2e_value, "unit": "unknowns/s", "h2d_bytes_per_step": unknowns * 8,
                "d2h_bytes_per_step": unknowns * 8},
        "roofline": roof,
        "clocks": clk.summary(),
    }

    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        Xs = X[:, :, :ORACLE_COLS].cpu().numpy()
        Fs = Fd[:, :, :ORACLE_COLS].cpu().numpy()
        Xr, t_or = _oracle_sample(A, B, C, Fs)
        line["cpu_baseline"] = {"value": N * M * ORACLE_COLS / t_or, "unit": "unknowns/s",
                                "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                                "sample": f"FP64 block-sweep oracle (numpy/LAPACK) on {ORACLE_COLS} of {K} columns"}
        line["rel_err_vs_oracle"] = oracle.rel_err(Xs, Xr)
        line["rel_res_sample"] = oracle.rel_res(A, B, C, Xs, Fs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    fac.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["f64", "f32", "tf32", "bf16", "bf16x3"], default="f64")
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows", type=int, default=N,
                    help="block rows N (smaller values only for profiler captures; the bench workload is 4096)")
    ap.add_argument("--segments", type=int, default=S, help="segments S (default 64)")
    args = ap.parse_args()
    global WORKLOAD
    globals()["N"], globals()["S"] = args.rows, args.segments
    WORKLOAD = f"acoustic PML operator N={args.rows} M={M} K={K} S={args.segments} (tridiag C, A=B=I)"
    if args.impl == "reference":
        return run_reference(args)
    import __graft_entry__

    __graft_entry__.build()
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
