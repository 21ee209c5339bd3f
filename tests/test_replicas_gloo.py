"""The multi-GPU path on CPU: two gloo ranks (world size 2).

With several GPUs the solve shards over right-hand-side columns: every rank
factors the same matrix and solves its own K columns, with no exchange on the
data path; the only collectives are the barrier and the maximum of the ranks'
times.  These tests run that host logic with gloo on the CPU: per-rank inputs,
independent per-rank solves (the oracle stands in for the GPU solve, which has
no multi-rank coupling), the slowest-rank time and the whole-job rate.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle
    from workloads import gen

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        N, M, K, S = 16, 8, 3, 4
        A, B, C = gen.acoustic_system(N, M)
        F = gen.acoustic_rhs(N, M, K, seed=bench.rank_seed(rank))
        X = oracle.solve_block_thomas(A, B, C, F)  # each rank's own columns, nothing exchanged
        t_local = 0.5 + rank  # rank 1 is the slowest
        t = bench.max_over_ranks(t_local, ws, torch.device("cpu"))
        rate = bench.job_rate(N * M * K, ws, t)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), F=F, X=X, t=t, rate=rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_columns(tmp_path):
    ws = 2
    port = _free_port()
    mp.start_processes(_rank_main, args=(ws, port, str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    # the slowest rank's time on both ranks, and the whole-job rate from it
    assert float(r0["t"]) == float(r1["t"]) == 1.5
    assert float(r0["rate"]) == float(r1["rate"]) == 16 * 8 * 3 * 2 / 1.5
    # distinct inputs per rank, each solved on its own
    assert not np.allclose(r0["F"], r1["F"])
    import oracle
    from workloads import gen

    A, B, C = gen.acoustic_system(16, 8)
    for r in (r0, r1):
        assert oracle.rel_res(A, B, C, r["X"], r["F"]) < 1e-13


def test_single_rank_needs_no_collective():
    import bench

    assert bench.max_over_ranks(2.5, 1, None) == 2.5
    assert bench.job_rate(100, 1, 2.0) == 50.0
