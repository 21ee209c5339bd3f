"""Adjoint gradients through the CUDA path (GPU only).

Bars: central finite differences in FP64 with step 1e-6 on an N=16, M=4, K=2
instance agree to 1e-6 relative; at full size (N=2048, M=64, K=128) every
gradient matches the FP64 oracle gradient (oracle/adjoint.py) to 1e-10
relative; the adjoint identity <G, P^{-1} F> = <P^{-T} G, F> holds.
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

    return bt


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def test_adjoint_dot_product_identity(bt):
    N, M, K, S = 48, 6, 3, 8
    A, B, C = gen.dominant_blocks(N, M, seed=4)
    F = gen.uniform_rhs(N, M, K, seed=5)
    G = gen.uniform_rhs(N, M, K, seed=6)
    with bt.factor(_t(A), _t(B), _t(C), S) as fac:
        X = fac.solve(_t(F))
        lam, _, _, _ = fac.adjoint(X, _t(G), want=("F",))
    lhs = float(torch.sum(_t(G) * X))
    rhs = float(torch.sum(lam * _t(F)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoint_matches_central_differences(bt):
    # L = 0.5 ||X - X_t||^2; L(+h) - L(-h) evaluated as 0.5 sum((X+ - X-)(X+ + X- - 2 X_t)).
    N, M, K, S = 16, 4, 2, 4
    A, B, C = gen.dominant_blocks(N, M, seed=13)
    F = gen.uniform_rhs(N, M, K, seed=20)
    Xt = gen.uniform_rhs(N, M, K, seed=14)
    Av, Bv, Cv, Fv = (_t(x).requires_grad_(True) for x in (A, B, C, F))
    X = bt.bt_solve(Av, Bv, Cv, Fv, S)
    loss = 0.5 * torch.sum((X - _t(Xt)) ** 2)
    loss.backward()
    grads = {"A": Av.grad.cpu().numpy(), "B": Bv.grad.cpu().numpy(), "C": Cv.grad.cpu().numpy(),
             "F": Fv.grad.cpu().numpy()}
    h = 1e-6
    rng = np.random.default_rng(0)
    checks = 0
    with torch.no_grad():
        for name in "ABCF":
            base = {"A": A, "B": B, "C": C, "F": F}
            for _ in range(10):
                idx = tuple(int(rng.integers(0, s)) for s in base[name].shape)
                if (name == "A" and idx[0] == 0) or (name == "B" and idx[0] == N - 1):
                    assert grads[name][idx] == 0.0
                    continue
                xs = []
                for sgn in (1, -1):
                    args = {k: v.copy() for k, v in base.items()}
                    args[name][idx] += sgn * h
                    with bt.factor(_t(args["A"]), _t(args["B"]), _t(args["C"]), S) as fac:
                        xs.append(fac.solve(_t(args["F"])).cpu().numpy())
                fd = 0.5 * float(np.sum((xs[0] - xs[1]) * (xs[0] + xs[1] - 2 * Xt))) / (2 * h)
                assert fd == pytest.approx(grads[name][idx], rel=1e-6, abs=1e-12), (name, idx)
                checks += 1
    assert checks >= 30


def test_adjoint_matches_oracle_gradient_full_size(bt):
    A, B, C, F, Xt = gen.config4()
    N, M, K = F.shape
    with bt.factor(_t(A), _t(B), _t(C), 64) as fac:
        X = fac.solve(_t(F))
        G = X - _t(Xt)
        dF, dA, dB, dC = fac.adjoint(X, G)
    Xn = X.cpu().numpy()
    rF, rA, rB, rC = oracle.adjoint_grads(A, B, C, Xn, Xn - Xt)
    for got, ref, name in ((dF, rF, "F"), (dA, rA, "A"), (dB, rB, "B"), (dC, rC, "C")):
        assert _rel(got.cpu().numpy(), ref) <= 1e-10, name
    assert float(dA[0].abs().max()) == 0.0 and float(dB[-1].abs().max()) == 0.0


def test_autograd_fp32_forward(bt):
    # FP32 inputs: the forward runs on FP64 factors and returns FP32, gradients come back in FP32.
    N, M, K, S = 64, 8, 4, 8
    A, B, C = gen.dominant_blocks(N, M, seed=2)
    F = gen.uniform_rhs(N, M, K, seed=3)
    Av, Bv, Cv = (_t(x).float().requires_grad_(True) for x in (A, B, C))
    Fv = _t(F).float().requires_grad_(True)
    X = bt.bt_solve(Av, Bv, Cv, Fv, S)
    assert X.dtype == torch.float32
    X.sum().backward()
    assert Av.grad.dtype == torch.float32 and Fv.grad.dtype == torch.float32
    Xr = oracle.solve_block_thomas(Av.detach().double().cpu().numpy(), Bv.detach().double().cpu().numpy(),
                                   Cv.detach().double().cpu().numpy(), Fv.detach().double().cpu().numpy())
    assert _rel(X.detach().double().cpu().numpy(), Xr) <= 1e-6


@pytest.mark.parametrize("precision", ["f32", "bf16x3"])
def test_autograd_fp32_forward_full_size(bt, precision):
    # The differentiation workload as specified: N = 2048, M = 64, K = 128,
    # L = 0.5 ||X - X_target||^2, the forward solve in FP32 arithmetic (FP32 CUDA
    # cores, or split-BF16 tensor cores) on FP64 factors with refinement, the
    # adjoint in FP64.  Against the FP64 oracle gradient at the oracle's own
    # solution: the forward's residual tolerance (1e-12) bounds the difference.
    A, B, C, F, Xt = gen.config4()
    Av, Bv, Cv, Fv = (_t(x).requires_grad_(True) for x in (A, B, C, F))
    X = bt.bt_solve(Av, Bv, Cv, Fv, 64, precision=precision, tol=1e-12)
    loss = 0.5 * torch.sum((X - _t(Xt)) ** 2)
    loss.backward()
    Xr = oracle.solve_block_thomas(A, B, C, F)
    assert oracle.rel_err(X.detach().cpu().numpy(), Xr) <= 1e-10
    rF, rA, rB, rC = oracle.adjoint_grads(A, B, C, Xr, Xr - Xt)
    for got, ref, name in ((Fv.grad, rF, "F"), (Av.grad, rA, "A"), (Bv.grad, rB, "B"), (Cv.grad, rC, "C")):
        assert _rel(got.cpu().numpy(), ref) <= 1e-8, name
    assert float(Av.grad[0].abs().max()) == 0.0 and float(Bv.grad[-1].abs().max()) == 0.0


def test_autograd_fp32_dtype_full_size(bt):
    # FP32 tensors in and out at full size: the gradients (FP32) against the
    # FP64 oracle gradient of the FP32-rounded inputs, to FP32 accuracy
    A, B, C, F, Xt = gen.config4()
    Av, Bv, Cv, Fv = (_t(x).float().requires_grad_(True) for x in (A, B, C, F))
    X = bt.bt_solve(Av, Bv, Cv, Fv, 64)
    assert X.dtype == torch.float32
    loss = 0.5 * torch.sum((X.double() - _t(Xt)) ** 2)
    loss.backward()
    A64, B64, C64, F64 = (v.detach().double().cpu().numpy() for v in (Av, Bv, Cv, Fv))
    Xr = oracle.solve_block_thomas(A64, B64, C64, F64)
    rF, rA, rB, rC = oracle.adjoint_grads(A64, B64, C64, Xr, Xr - Xt)
    for got, ref, name in ((Fv.grad, rF, "F"), (Av.grad, rA, "A"), (Bv.grad, rB, "B"), (Cv.grad, rC, "C")):
        assert got.dtype == torch.float32
        assert _rel(got.double().cpu().numpy(), ref) <= 1e-6, name
