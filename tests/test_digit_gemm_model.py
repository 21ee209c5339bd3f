"""Pins of the digit-slice block product (csrc/gemm_digits.cu) on the CPU.

The method: every contraction index k is balanced, X[:, k] 2^t_k and
2^-t_k Y[k, :] with t_k = floor((ry(k) - cx(k)) / 2) from the exponents of the
column maxima of X and the row maxima of Y (an index whose column or row is
zero is dropped); a balanced x with max_k |x| < 2^ex is taken in fixed point
f = round(x 2^(56 - ex)) and written as 8 balanced base-128 digits; likewise Y's
columns; the 36 digit pairs with p + q <= 7 are summed per level p + q (each
level an exact FP32 sum on the tensor cores), and the levels are combined as
hi 2^28 + lo with one rounding, scaled by 2^(ex + ey - 63).  Here every step
is carried out in exact integer arithmetic and compared with the exact
rational product: the digits' ranges, the exactness of every level sum in FP32
(|c_d| < 2^24 for M = 128), and the stated bound
|D - sum_k X[r][k] Y[k][c]| <= M 2^(ex(r) + ey(c) - 52).  Scaling the
contraction index by powers of two (X D, D^-1 Y) leaves the result unchanged,
so a system whose unknowns span many binades keeps FP64-level products.
Planted mistakes (a dropped level, a wrong level weight, a transposed operand,
the balancing applied to one side only) break the bound.
"""

import math
from fractions import Fraction

import numpy as np

M = 128
GD = 8
FB = 56


def _exp(amax):
    return math.frexp(amax)[1] if amax > 0 else 0


def _floor_log2(v):
    return math.frexp(abs(v))[1] - 1 if v != 0 else None


def _balance(X, Y):
    """t_k (None: the index is dropped) from the exponents of max_r |X[r][k]|
    and max_c |Y[k][c]|."""
    t = []
    for k in range(M):
        a = max((_floor_log2(v) for v in X[:, k] if v != 0), default=None)
        b = max((_floor_log2(v) for v in Y[k, :] if v != 0), default=None)
        t.append(None if a is None or b is None else (b - a) // 2)
    return t


def _digits(x, e):
    f = round(Fraction(x) * Fraction(2) ** (FB - e))  # nearest, ties to even
    f = int(f)
    d = [0] * GD
    for p in range(GD - 1, 0, -1):
        r = ((f + 64) & 127) - 64
        d[p] = r
        f = (f - r) >> 7
    d[0] = f
    return d


def _product(X, Y, rows, cols, drop_level=None, weight=128, transpose_y=False, one_sided=False):
    Yu = Y.T if transpose_y else Y
    t = _balance(X, Yu)
    # balanced operands, exact (powers of two; dropped indices as zeros)
    Xb = [[Fraction(0) if t[k] is None else Fraction(float(X[r, k])) * Fraction(2) ** t[k] for k in range(M)]
          for r in range(M)]
    Yb = [[Fraction(0) if t[k] is None else Fraction(float(Yu[k, c])) * (1 if one_sided else Fraction(2) ** -t[k])
           for c in range(M)] for k in range(M)]
    ex = {r: _exp(max(abs(v) for v in Xb[r])) for r in rows}
    ey = {c: _exp(max(abs(Yb[k][c]) for k in range(M))) for c in cols}
    xd = {r: [_digits(Xb[r][k], ex[r]) for k in range(M)] for r in rows}
    yd = {c: [_digits(Yb[k][c], ey[c]) for k in range(M)] for c in cols}
    out, levels = {}, []
    for r in rows:
        for c in cols:
            cd = [0] * GD
            for p in range(GD):
                for q in range(GD - p):
                    cd[p + q] += sum(xd[r][k][p] * yd[c][k][q] for k in range(M))
            if drop_level is not None:
                cd[drop_level] = 0
            levels.extend(cd)
            hi = ((cd[0] * weight + cd[1]) * 128 + cd[2]) * 128 + cd[3]
            lo = ((cd[4] * 128 + cd[5]) * 128 + cd[6]) * 128 + cd[7]
            t = float(hi * 2 ** 28 + lo)  # one rounding, as fma(hi, 2^28, lo)
            # level d weighs 128^(14 - d) 2^(ex + ey - 112): T 2^(ex + ey - 63)
            out[r, c] = (math.ldexp(t, ex[r] + ey[c] - 2 * FB + 7 * (GD - 1)), ex[r], ey[c])
    return out, levels, xd, yd


def _inputs(seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((M, M)) * np.exp2(rng.integers(-20, 20, (M, 1)))
    Y = rng.standard_normal((M, M)) * np.exp2(rng.integers(-20, 20, (1, M)))
    X[3] = 0.0                       # a zero row
    X[5, 7:] *= 2.0 ** -40           # a row with one large entry
    Y[:, 9] *= 2.0 ** -1000          # a column near the bottom of the range
    return X, Y


def _exact(X, Y, r, c):
    return sum(Fraction(float(X[r, k])) * Fraction(float(Y[k, c])) for k in range(M))


ROWS, COLS = [0, 3, 5, 77, 127], [0, 9, 64, 100]


def test_digits_levels_and_bound():
    X, Y = _inputs(1)
    Y[11, :] = 0.0                   # a dropped contraction index
    out, levels, xd, yd = _product(X, Y, ROWS, COLS)
    for dig in list(xd.values()) + list(yd.values()):
        for d in dig:
            assert abs(d[0]) <= 128 and all(abs(v) <= 64 for v in d[1:])
    assert max(abs(v) for v in levels) < 2 ** 24  # every level sum is exact in FP32
    for (r, c), (v, er, ec) in out.items():
        err = abs(Fraction(v) - _exact(X, Y, r, c))
        assert err <= M * Fraction(2) ** (er + ec - 52), (r, c, float(err))
    # the bound is FP64-level against the product's scale
    for (r, c), (v, er, ec) in out.items():
        scale = M * float(np.max(np.abs(X[r]))) * float(np.max(np.abs(Y[:, c])))
        if scale > 0:
            assert abs(v - float(_exact(X, Y, r, c))) <= 2.0 ** -49 * scale


def test_contraction_scaling_leaves_the_product_unchanged():
    # X D and D^-1 Y with D powers of two over 2^-300 .. 2^300 (the unknowns of
    # a block row scaled): every digit and every result is the same, so the
    # error stays at the unscaled product's FP64 level although the rows of
    # X D span 600 binades
    X, Y = _inputs(3)
    Y[:, 9] *= 2.0 ** 1000           # (2^-1300 would not be representable)
    d = np.exp2(np.random.default_rng(4).integers(-300, 301, M)).astype(np.float64)
    rows, cols = [0, 5, 77], [0, 9, 100]
    out, _, xd, yd = _product(X, Y, rows, cols)
    out2, _, xd2, yd2 = _product(X * d[None, :], Y / d[:, None], rows, cols)
    assert xd == xd2 and yd == yd2
    assert {k: v[0] for k, v in out.items()} == {k: v[0] for k, v in out2.items()}
    for (r, c), (v, er, ec) in out.items():
        scale = M * float(np.max(np.abs(X[r]))) * float(np.max(np.abs(Y[:, c])))
        assert abs(v - float(_exact(X, Y, r, c))) <= 2.0 ** -47 * scale


def test_level_sums_stay_exact_at_the_worst_case():
    # every digit at its largest magnitude: the level sums reach their bound
    worst = [128] + [64] * (GD - 1)
    for d in range(GD):
        s = M * sum(worst[p] * worst[d - p] for p in range(d + 1))
        assert s < 2 ** 24, (d, s)


def test_planted_mistakes_break_the_bound():
    X, Y = _inputs(2)
    rows, cols = [0, 77], [0, 100]

    def violates(**kw):
        out, _, _, _ = _product(X, Y, rows, cols, **kw)
        return any(abs(Fraction(v) - _exact(X, Y, r, c)) > M * Fraction(2) ** (er + ec - 52)
                   for (r, c), (v, er, ec) in out.items())

    assert not violates()
    assert violates(drop_level=5)
    assert violates(weight=64)
    assert violates(transpose_y=True)
    assert violates(one_sided=True)
