"""Refined batches (bt_batch_* with a mixed precision) vs the CPU oracle (GPU only).

The sets of each factored matrix are packed into one panel (each scaled by a
power of two), refined as one solve per matrix until every set meets the
tolerance on its own, and unpacked; the whole plan is one CUDA graph.  Bars:
every set meets the requested relative residual ||F_s - P X_s|| / ||F_s|| <=
tol on its own -- also a set whose scale is 1e-30 or 1e25 times its
neighbours' -- and matches the FP64 oracle column by column within 1e-10 (the
refined paths' bar).
"""

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


def _check_sets(mats, which, Fs_np, Xs, tol):
    for i, (F, X) in enumerate(zip(Fs_np, Xs)):
        A, B, C = mats[which[i]]
        Xn = X.cpu().numpy()
        if not np.any(F):
            assert not np.any(Xn), i
            continue
        # the per-set guarantee, recomputed by the oracle in FP64 (1 % for the
        # library's own residual error: the double-word residual of stencils)
        assert oracle.rel_res(A, B, C, Xn, F) <= tol * 1.01, i
        Xr = oracle.solve_block_thomas(A, B, C, F)
        assert oracle.rel_err(Xn, Xr) <= 1e-10, i
        assert oracle.col_err(Xn, Xr) <= 1e-10, i


def _uneven_sets(N, M, Ks, seed0):
    Fs = [gen.uniform_rhs(N, M, k, seed=seed0 + i) for i, k in enumerate(Ks)]
    Fs[1] = Fs[1] * 1e-30  # scales far apart: the packing rescales each set
    Fs[3] = Fs[3] * 1e25
    Fs[4] = np.zeros_like(Fs[4])  # a zero set stays zero
    return Fs


@pytest.mark.parametrize("precision,M", [("bf16x3", 64), ("tf32", 64), ("f32", 24)])
def test_refined_plan_every_set_meets_its_tolerance(bt, precision, M):
    N, tol = 64, 1e-11
    mats = [gen.dominant_blocks(N, M, seed=s) for s in (41, 42)]
    Ks = [3, 130, 17, 64, 5, 1, 129]
    which = [0, 1, 0, 1, 0, 1, 1]
    Fs_np = _uneven_sets(N, M, Ks, 60)
    with bt.factor(*(_t(a) for a in mats[0]), 8) as f0, bt.factor(*(_t(a) for a in mats[1]), 16) as f1:
        facs = [(f0, f1)[w] for w in which]
        Fs = [_t(F) for F in Fs_np]
        Xs = [torch.full_like(F, np.nan) for F in Fs]
        plan = bt.BatchPlan(facs, Fs, Xs, precision=precision, tol=tol)
        assert plan.items == 2 and plan.graph == 1
        for rnd in range(2):
            if rnd == 1:  # new values in the same buffers: the replay reads them
                Fs_np[2] = gen.uniform_rhs(N, M, Ks[2], seed=99)
                Fs[2].copy_(_t(Fs_np[2]))
            plan.run()
            plan.status()
            _check_sets(mats, which, Fs_np, Xs, tol)
            for i in range(len(Ks)):
                inf = plan.info(i)
                assert inf["converged"]
        plan.close()


def test_refined_plan_recaptures_after_the_handle_grows(bt):
    # a later, wider solve on a plan's handle reallocates its refinement
    # scratch: the next run prepares and captures the plan again
    N, M, tol = 64, 64, 1e-11
    mats = [gen.dominant_blocks(N, M, seed=7)]
    Ks = [2, 40, 9, 33, 4]
    Fs_np = _uneven_sets(N, M, Ks, 80)
    with bt.factor(*(_t(a) for a in mats[0]), 8) as fac:
        Fs = [_t(F) for F in Fs_np]
        Xs = [torch.empty_like(F) for F in Fs]
        plan = bt.BatchPlan([fac] * len(Ks), Fs, Xs, precision="bf16x3", tol=tol)
        plan.run()
        plan.status()
        _check_sets(mats, [0] * len(Ks), Fs_np, Xs, tol)
        Fw = gen.uniform_rhs(N, M, 700, seed=3)
        Xw = fac.solve(_t(Fw), precision="bf16x3", tol=tol)
        assert oracle.col_err(Xw.cpu().numpy(), oracle.solve_block_thomas(*mats[0], Fw)) <= 1e-10
        for X in Xs:
            X.zero_()
        plan.run()
        plan.status()
        _check_sets(mats, [0] * len(Ks), Fs_np, Xs, tol)
        plan.close()


def test_refined_plan_unit_stencil(bt):
    # acoustic-style unit stencils (M = 128): the split-BF16 panel flow with the
    # double-word residual inside the plan's graph
    N, M, S, tol = 64, 128, 8, 1e-11
    mats = [gen.acoustic_system(N, M)]
    Ks = [40, 1, 200, 7, 3]
    Fs_np = [gen.acoustic_rhs(N, M, k, seed=20 + i) for i, k in enumerate(Ks)]
    Fs_np[1] = Fs_np[1] * 1e-30
    Fs_np[3] = Fs_np[3] * 1e25
    Fs_np[4] = np.zeros_like(Fs_np[4])
    with bt.factor(*(_t(a) for a in mats[0]), S) as fac:
        Fs = [_t(F) for F in Fs_np]
        Xs = [torch.empty_like(F) for F in Fs]
        plan = bt.BatchPlan([fac] * len(Ks), Fs, Xs, precision="bf16x3", tol=tol)
        for _ in range(2):
            plan.run()
            plan.status()
            _check_sets(mats, [0] * len(Ks), Fs_np, Xs, tol)
        plan.close()


def test_refined_plan_config3_shape_sampled(bt):
    # the uneven-set workload at full matrix size (N = 2048, M = 64, four
    # matrices), 16 of its 64 sets: one column from every 128-column tile and
    # the last column of each set against the oracle.  The refinement holds the
    # residual; a column's forward error can exceed it by the conditioning, so
    # a 1e-10 error bar takes tol 1e-11 (as in the other refined tests)
    mats, sets = gen.config3(n_sets=16)
    facs = [bt.factor(*(_t(a) for a in m), 64) for m in mats]
    Fs = [_t(s.F) for s in sets]
    Xs = [torch.empty_like(F) for F in Fs]
    plan = bt.BatchPlan([facs[s.matrix] for s in sets], Fs, Xs, precision="bf16x3", tol=1e-11)
    assert plan.items == 4
    plan.run()
    plan.status()
    rng = np.random.default_rng(0)
    for i, (st, X) in enumerate(zip(sets, Xs)):
        assert plan.info(i)["converged"]
        cols = sorted({int(t + rng.integers(0, min(128, st.K - t))) for t in range(0, st.K, 128)} | {st.K - 1})
        A, B, C = mats[st.matrix]
        Xr = oracle.solve_block_thomas(A, B, C, st.F[:, :, cols])
        assert oracle.col_err(X[:, :, cols].cpu().numpy(), Xr) <= 1e-10, (i, st.K)
    plan.close()
    for f in facs:
        f.close()


def test_refined_plan_arguments(bt):
    N, M = 32, 64
    mats = [gen.dominant_blocks(N, M, seed=1)]
    with bt.factor(*(_t(a) for a in mats[0]), 4) as fac:
        F = _t(gen.uniform_rhs(N, M, 3, seed=2))
        X = torch.empty_like(F)
        plan = bt.BatchPlan([fac], [F], [X], precision="bf16x3", tol=1e-11)
        with pytest.raises(bt.BtError) as ei:
            plan.info(0)  # before bt_batch_status
        assert ei.value.name == "BT_ERR_ARG"
        with pytest.raises(bt.BtError) as ei:
            plan.debug(limit_s=1.0)  # no grid barrier in a refined plan
        assert ei.value.name == "BT_ERR_UNSUPPORTED"
        plan.run()
        plan.status()
        with pytest.raises(bt.BtError) as ei:
            plan.info(1)
        assert ei.value.name == "BT_ERR_ARG"
        plan.close()
    # the tensor-core precisions refuse block sizes past the largest tile, as bt_solve_ex does
    with bt.factor(*(_t(a) for a in gen.dominant_blocks(8, 150, seed=1)), 4) as f150:
        F = _t(gen.uniform_rhs(8, 150, 3, seed=2))
        with pytest.raises(bt.BtError) as ei:
            bt.BatchPlan([f150], [F], [torch.empty_like(F)], precision="bf16x3")
        assert ei.value.name == "BT_ERR_UNSUPPORTED"
