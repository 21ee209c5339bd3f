"""Batched FP64 solves (bt_batch_*, bt_solve_batched) vs the CPU oracle (GPU only).

Many right-hand-side sets of uneven K against several factored matrices run
as one persistent launch replayed from a CUDA graph.  Every set must match the
FP64 oracle to 1e-12 relative error, the bar of the plain FP64 method.
"""

import numpy as np
import pytest

import oracle
from workloads import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
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


def _factors(bt, mats, Ss):
    return [bt.factor(_t(A), _t(B), _t(C), S) for (A, B, C), S in zip(mats, Ss)]


def _check(mats, sets, Xs):
    for st, X in zip(sets, Xs):
        A, B, C = mats[st.matrix]
        Xr = oracle.solve_block_thomas(A, B, C, st.F)
        err = oracle.rel_err(X.cpu().numpy(), Xr)
        assert err <= TOL, (st.K, err)
        assert oracle.col_err(X.cpu().numpy(), Xr) <= TOL, st.K


@pytest.mark.parametrize("S_list", [(8, 16, 4), (1, 64, 2)])
def test_batched_uneven_sets_match_oracle(bt, S_list):
    # three matrices with different segment counts (S = 1 and S = N included),
    # eleven sets with K from 1 to 70 (several column tiles, ragged tails)
    N, M = 64, 8
    mats = [gen.dominant_blocks(N, M, seed) for seed in (1, 2, 3)]
    Ks = [1, 2, 3, 5, 8, 9, 17, 33, 64, 70, 4]
    sets = [gen.RhsSet(matrix=i % 3, K=k, F=gen.uniform_rhs(N, M, k, seed=50 + i)) for i, k in enumerate(Ks)]
    facs = _factors(bt, mats, S_list)
    Fs = [_t(s.F) for s in sets]
    Xs = bt.solve_batched([facs[s.matrix] for s in sets], Fs)
    torch.cuda.synchronize()
    _check(mats, sets, Xs)


def test_batched_plan_replays_graph(bt):
    # a plan is built once and replayed; new values in the same F buffers give
    # new solutions, and the launch is a single persistent cooperative kernel
    N, M = 128, 16
    mats = [gen.dominant_blocks(N, M, seed) for seed in (4, 5)]
    Ks = [7, 40, 1, 129]
    sets = [gen.RhsSet(matrix=i % 2, K=k, F=gen.uniform_rhs(N, M, k, seed=70 + i)) for i, k in enumerate(Ks)]
    facs = _factors(bt, mats, (16, 32))
    Fs = [_t(s.F) for s in sets]
    Xs = [torch.empty_like(F) for F in Fs]
    plan = bt.BatchPlan([facs[s.matrix] for s in sets], Fs, Xs)
    assert plan.graph == 1
    assert plan.items > 0 and plan.stages >= 3 and plan.ctas >= 1
    plan.run()
    plan.status()
    _check(mats, sets, Xs)
    sets2 = [gen.RhsSet(matrix=s.matrix, K=s.K, F=gen.uniform_rhs(N, M, s.K, seed=90 + i)) for i, s in enumerate(sets)]
    for F, s in zip(Fs, sets2):
        F.copy_(_t(s.F))
    for _ in range(3):
        plan.run()
    plan.status()
    _check(mats, sets2, Xs)
    plan.close()


@pytest.mark.parametrize("k_tile", [4, 16, 32])
def test_batched_tile_choices(bt, k_tile):
    N, M = 64, 16
    mats = [gen.dominant_blocks(N, M, 9)]
    sets = [gen.RhsSet(matrix=0, K=k, F=gen.uniform_rhs(N, M, k, seed=k)) for k in (3, 31, 45)]
    facs = _factors(bt, mats, (8,))
    Xs = bt.solve_batched([facs[0]] * 3, [_t(s.F) for s in sets], k_tile=k_tile)
    torch.cuda.synchronize()
    _check(mats, sets, Xs)


def test_batched_config3_shape_sampled(bt):
    # the uneven-set workload at full matrix size (N = 2048, M = 64, four
    # matrices); 16 of its 64 sets, checked on sampled columns
    mats, sets = gen.config3(n_sets=16)
    facs = _factors(bt, mats, (64, 64, 64, 64))
    Fs = [_t(s.F) for s in sets]
    Xs = bt.solve_batched([facs[s.matrix] for s in sets], Fs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for st, X in zip(sets, Xs):
        # one column from every 128-column tile, and the last column
        cols = sorted({int(t + rng.integers(0, min(128, st.K - t))) for t in range(0, st.K, 128)} | {st.K - 1})
        A, B, C = mats[st.matrix]
        Xr = oracle.solve_block_thomas(A, B, C, st.F[:, :, cols])
        err = oracle.rel_err(X[:, :, cols].cpu().numpy(), Xr)
        assert err <= TOL, (st.K, err)
        assert oracle.col_err(X[:, :, cols].cpu().numpy(), Xr) <= TOL, st.K


def test_batched_rejects_bad_input(bt):
    N = 32
    f8 = bt.factor(*(_t(a) for a in gen.dominant_blocks(N, 8, 1)), 4)
    f4 = bt.factor(*(_t(a) for a in gen.dominant_blocks(N, 4, 1)), 4)
    F8 = _t(gen.uniform_rhs(N, 8, 3, seed=1))
    F4 = _t(gen.uniform_rhs(N, 4, 3, seed=1))
    with pytest.raises(bt.BtError) as e:
        bt.solve_batched([f8, f4], [F8, F4])  # block sizes differ
    assert e.value.name == "BT_ERR_ARG"
    with pytest.raises(bt.BtError) as e:
        bt.solve_batched([f8, f8], [F8, F8], [F8, torch.empty_like(F8)])  # X overlaps F
    assert e.value.name == "BT_ERR_ARG"
    X = torch.empty_like(F8)
    with pytest.raises(bt.BtError) as e:
        bt.solve_batched([f8, f8], [F8, torch.empty_like(F8)], [X, X])  # two outputs share memory
    assert e.value.name == "BT_ERR_ARG"


def test_batched_matrices_of_different_sizes(bt):
    # one launch over sets whose matrices differ in N and S (same block size)
    M = 8
    mats = [gen.dominant_blocks(48, M, 11), gen.dominant_blocks(96, M, 12)]
    facs = _factors(bt, mats, (6, 32))
    sets = [gen.RhsSet(matrix=0, K=5, F=gen.uniform_rhs(48, M, 5, seed=1)),
            gen.RhsSet(matrix=1, K=19, F=gen.uniform_rhs(96, M, 19, seed=2)),
            gen.RhsSet(matrix=0, K=1, F=gen.uniform_rhs(48, M, 1, seed=3))]
    Xs = bt.solve_batched([facs[s.matrix] for s in sets], [_t(s.F) for s in sets])
    torch.cuda.synchronize()
    _check(mats, sets, Xs)


def test_grid_barrier_timeout_is_reported_and_the_plan_recovers(bt):
    # Failure detection without a GPU fault: CTA 0 of the persistent launch
    # leaves instead of arriving at the barrier after the first stage, so the
    # other CTAs' bounded waits (limited to 5 ms here) run out; the run reports
    # BT_ERR_TIMEOUT promptly, and the same plan then solves correctly.
    import time

    mats = [gen.dominant_blocks(64, 16, seed=s) for s in (1, 2)]
    sets = [gen.uniform_rhs(64, 16, k, seed=10 + k) for k in (5, 40)]
    facs = _factors(bt, mats, (8, 16))
    Fs = [_t(F) for F in sets]
    Xs = [torch.zeros_like(F) for F in Fs]
    plan = bt.BatchPlan(facs, Fs, Xs)
    assert plan.stages >= 2 and plan.ctas >= 2
    plan.debug(limit_s=0.005, skip_stage=0)
    t0 = time.perf_counter()
    plan.run()
    with pytest.raises(bt.BtError) as ei:
        plan.status()
    assert ei.value.name == "BT_ERR_TIMEOUT"
    assert time.perf_counter() - t0 < 2.0  # the limit, not the 20 s default
    # the failure was contained: the device and the plan still work
    plan.debug(limit_s=0.0, skip_stage=-1)
    plan.run()
    plan.status()
    for (A, B, C), F, X in zip(mats, sets, Xs):
        Xr = oracle.solve_block_thomas(A, B, C, F)
        assert oracle.rel_err(X.cpu().numpy(), Xr) <= TOL
        assert oracle.col_err(X.cpu().numpy(), Xr) <= TOL
    plan.close()
    for f in facs:
        f.close()


def test_batch_debug_rejects_bad_arguments(bt):
    mats = [gen.dominant_blocks(16, 4, seed=1)]
    facs = _factors(bt, mats, (4,))
    F = _t(gen.uniform_rhs(16, 4, 3, seed=2))
    plan = bt.BatchPlan(facs, [F], [torch.zeros_like(F)])
    for lim, skip in ((-1.0, -1), (61.0, -1), (0.0, -2)):
        with pytest.raises(bt.BtError) as ei:
            plan.debug(limit_s=lim, skip_stage=skip)
        assert ei.value.name == "BT_ERR_ARG"
    plan.close()
    facs[0].close()
