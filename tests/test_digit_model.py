"""CPU model of the exact digit residual (the method behind bt_residual "digits"),
in exact integer arithmetic, checked against the oracle's residual F - P X.

The model follows the method's definition, not the CUDA code: scales e_A(j,m)
over row m of A_j, B_j, C_j and e_X(n) over column n of X; balanced base-128
digits of round(v 2^(49-e)); per-diagonal sums of the 28 digit-pair products
with p + q <= 6; T = sum_d c_d 128^(6-d); r = round(F / u) + T in units
u = 2^(e_A + e_X - 56).  Checked here: the stated bound |r - r_exact| <=
7.5 M 2^(e_A + e_X - 49) on random, near-solution and adversarial inputs; the
digit and accumulator bounds that make FP32 accumulation exact; that the
64-bit sum taken modulo 2^64 recovers r while |r| < 2^63 u; and that planted
mistakes (a dropped digit pair, six digits, a sign slip on C) break the bound.
"""

import math

import numpy as np
import pytest

import oracle
from workloads import gen

ND, FB = 7, 49


def _scale(mx: float) -> int:
    return math.frexp(mx)[1] if mx > 0 else 0


def _digits(v: float, e: int, nd: int = ND):
    """Balanced base-128 digits, most significant first, of round(v 2^(7 nd - e))."""
    x = math.ldexp(abs(v), 7 * nd - e)  # exact (power-of-two scaling)
    f = int(math.floor(x + 0.5))
    if v < 0:
        f = -f
    d = [0] * nd
    for p in range(nd - 1, 0, -1):
        t = ((f + 64) & 127) - 64
        d[p] = t
        f = (f - t) >> 7
    d[0] = f
    return d


def _round_to_unit(v: float, u: int) -> int:
    """round(v / 2^u) to an integer (half away from zero), exactly."""
    x = math.ldexp(abs(v), -u)
    r = int(math.floor(x + 0.5))
    return -r if v < 0 else r


def residual_model(A, B, C, X, F, nd=ND, drop_pair=None, c_sign=-1.0):
    """r = F + A_j X_{j-1} + B_j X_{j+1} - C_j X_j by the digit method (exact integers)."""
    N, M, K = X.shape
    blocks = [(A, -1), (B, +1), (c_sign * C, 0)]  # (operator block, neighbour offset)
    ea = [[_scale(max(np.abs(A[j, m]).max(), np.abs(B[j, m]).max(), np.abs(C[j, m]).max()))
           for m in range(M)] for j in range(N)]
    ex = [_scale(np.abs(X[:, :, n]).max()) for n in range(K)]
    xd = {(j, k, n): _digits(X[j, k, n], ex[n], nd) for j in range(N) for k in range(M) for n in range(K)}
    R = np.zeros_like(F)
    acc_max = 0
    for j in range(N):
        for m in range(M):
            ad = [[_digits(blk[j, m, k], ea[j][m], nd) for k in range(M)] for blk, _ in blocks]
            for n in range(K):
                c = [0] * nd
                for b, (_, off) in enumerate(blocks):
                    jx = j + off
                    if jx < 0 or jx >= N:
                        continue
                    for k in range(M):
                        a, x = ad[b][k], xd[(jx, k, n)]
                        for p in range(nd):
                            for q in range(nd - p):
                                if drop_pair == (p, q):
                                    continue
                                c[p + q] += a[p] * x[q]
                acc_max = max(acc_max, max(abs(v) for v in c))
                T = 0
                for d in range(nd):
                    T = T * 128 + c[d]
                u = ea[j][m] + ex[n] - (14 + 7 * (nd - 1))
                Rfix = _round_to_unit(F[j, m, n], u) + T
                R[j, m, n] = math.ldexp(float(Rfix), u)
    return R, acc_max


def _bound(A, B, C, X):
    M = C.shape[1]
    ea = np.array([[_scale(max(np.abs(A[j, m]).max(), np.abs(B[j, m]).max(), np.abs(C[j, m]).max()))
                    for m in range(M)] for j in range(C.shape[0])])
    ex = np.array([_scale(np.abs(X[:, :, n]).max()) for n in range(X.shape[2])])
    return 7.5 * M * np.ldexp(1.0, ea[:, :, None] + ex[None, None, :] - 49)


def _case(kind, N=3, M=8, K=3):
    rng = np.random.default_rng(5)
    A, B, C = gen.dominant_blocks(N, M, seed=N + M)
    F = gen.uniform_rhs(N, M, K, seed=2)
    if kind == "random":
        X = gen.uniform_rhs(N, M, K, seed=3)
    elif kind == "near":
        X = oracle.solve_block_thomas(A, B, C, F) * (1 + 1e-7 * rng.standard_normal((N, M, K)))
    else:  # adversarial: every entry positive and near its maximum, F = P X + small
        A = rng.uniform(0.75, 1.0, (N, M, M))
        B = rng.uniform(0.75, 1.0, (N, M, M))
        C = -rng.uniform(0.75, 1.0, (N, M, M))
        A[0] = 0.0
        B[N - 1] = 0.0
        X = rng.uniform(0.75, 1.0, (N, M, K))
        F = oracle.apply_P(A, B, C, X) + rng.uniform(-1e-6, 1e-6, (N, M, K))
    return A, B, C, X, F


@pytest.mark.parametrize("kind", ["random", "near", "adversarial"])
def test_model_within_bound(kind):
    A, B, C, X, F = _case(kind)
    R, acc_max = residual_model(A, B, C, X, F)
    err = np.abs(R - oracle.residual(A, B, C, X, F))
    assert (err <= _bound(A, B, C, X)).all(), float((err / _bound(A, B, C, X)).max())
    assert acc_max < 2 ** 24


def test_digits_reconstruct_and_stay_small():
    rng = np.random.default_rng(9)
    for _ in range(2000):
        e = int(rng.integers(-40, 40))
        v = float(rng.uniform(-1, 1)) * 2.0 ** e * (1 - 2 ** -52)
        d = _digits(v, e)
        assert abs(d[0]) <= 128 and all(abs(t) <= 64 for t in d[1:])
        val = sum(math.ldexp(d[p], e - 7 * (p + 1)) for p in range(ND))
        assert abs(val - v) <= math.ldexp(1.0, e - 50)


def test_accumulator_bound_admits_fp32():
    # worst case of one diagonal sum: 2 pairs with one leading digit (128 x 64),
    # the others 64 x 64, over 3M contraction terms -- below 2^24 for M <= 128
    for M in (64, 128):
        worst = max(3 * M * (2 * 128 * 64 + max(0, d - 1) * 64 * 64) if d > 0 else 3 * M * 128 * 128
                    for d in range(ND))
        assert worst < 2 ** 24, (M, worst)
    assert 3 * 256 * (2 * 128 * 64 + 5 * 64 * 64) >= 2 ** 24  # M = 256 would not be exact


def test_sum_modulo_2_64_recovers_the_residual():
    rng = np.random.default_rng(3)
    for _ in range(1000):
        T = int(rng.integers(-2 ** 62, 2 ** 62)) * int(rng.integers(1, 16))  # may exceed 2^63
        R = int(rng.integers(-2 ** 62, 2 ** 62))
        Ffix = R - T
        s = ((Ffix % 2 ** 64) + (T % 2 ** 64)) % 2 ** 64
        if s >= 2 ** 63:
            s -= 2 ** 64
        assert s == R


@pytest.mark.parametrize("mistake", ["drop_00", "drop_22", "six_digits", "c_sign"])
def test_planted_mistakes_break_the_bound(mistake):
    A, B, C, X, F = _case("near")
    kw = {"drop_00": dict(drop_pair=(0, 0)), "drop_22": dict(drop_pair=(2, 2)),
          "six_digits": dict(nd=6), "c_sign": dict(c_sign=1.0)}[mistake]
    R, _ = residual_model(A, B, C, X, F, **kw)
    err = np.abs(R - oracle.residual(A, B, C, X, F))
    assert (err > _bound(A, B, C, X)).any()
