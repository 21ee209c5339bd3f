"""Autotuner of the segment count and tile (GPU only): it must pick one of the
candidates it timed, and the factorizations it hands back must solve."""

import numpy as np
import pytest

import oracle
from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def bt():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1108_4181_gb300 as bt

    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    return bt


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_tune_batched_picks_a_timed_candidate(bt):
    from paper_1108_4181_gb300 import tune

    N, M = 128, 16
    mats_np = [gen.dominant_blocks(N, M, s) for s in (1, 2)]
    mats = [tuple(_t(a) for a in m) for m in mats_np]
    Ks = [3, 17, 40, 1]
    sets_np = [gen.RhsSet(matrix=i % 2, K=k, F=gen.uniform_rhs(N, M, k, seed=i)) for i, k in enumerate(Ks)]
    sets = [(s.matrix, _t(s.F)) for s in sets_np]
    res = tune.tune_batched(mats, sets, S_candidates=(4, 8, 16, 3, 256), tiles=(0, 8), reps=2)
    assert res.S in (4, 8, 16)  # 3 and 256 do not divide / exceed N
    assert (res.S, res.k_tile) in res.table
    assert res.ms == min(res.table.values())
    assert {S for S, _ in res.table} == {4, 8, 16}
    Xs = bt.solve_batched([res.factors[i] for i, _ in sets], [F for _, F in sets], k_tile=res.k_tile)
    torch.cuda.synchronize()
    for st, X in zip(sets_np, Xs):
        A, B, C = mats_np[st.matrix]
        assert oracle.rel_err(X.cpu().numpy(), oracle.solve_block_thomas(A, B, C, st.F)) <= 1e-12
    for f in res.factors:
        f.close()


def test_tune_solve_mixed(bt):
    from paper_1108_4181_gb300 import tune

    N, M, K = 256, 64, 96
    A, B, C = gen.acoustic_system(N, M)
    F = gen.acoustic_rhs(N, M, K, seed=3)
    res = tune.tune_solve(_t(A), _t(B), _t(C), _t(F), precision="bf16x3", tol=1e-10,
                          S_candidates=(8, 16, 32), reps=2)
    assert res.S in (8, 16, 32) and len(res.table) == 3
    X, info = res.factors[0].solve(_t(F), precision="bf16x3", tol=1e-10, return_info=True)
    assert info["converged"]
    assert oracle.rel_res(A, B, C, X.cpu().numpy(), F) <= 1e-10
    res.factors[0].close()


def test_tune_batched_refined_picks_a_timed_candidate(bt):
    from paper_1108_4181_gb300 import tune

    N, M = 128, 64
    mats_np = [gen.dominant_blocks(N, M, s) for s in (3, 4)]
    mats = [tuple(_t(a) for a in m) for m in mats_np]
    sets_np = [gen.RhsSet(matrix=i % 2, K=k, F=gen.uniform_rhs(N, M, k, seed=20 + i)) for i, k in enumerate((5, 130))]
    sets = [(s.matrix, _t(s.F)) for s in sets_np]
    res = tune.tune_batched_refined(mats, sets, tol=1e-11, S_candidates=(8, 16, 3), reps=1)
    assert res.S in (8, 16) and res.ms == min(res.table.values())
    assert {S for S, _ in res.table} == {8, 16}
    for st in sets_np:
        A, B, C = mats_np[st.matrix]
        X = res.factors[st.matrix].solve(_t(st.F), precision="bf16x3", tol=1e-11).cpu().numpy()
        assert oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, st.F)) <= 1e-10
    for f in res.factors:
        f.close()
