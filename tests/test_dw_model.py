"""CPU model of the FP32 double-word stencil residual (bt_residual method 3, the
refinement residual of unit-stencil operators), checked against the exact
residual.

The model follows the method's definition, not the CUDA code:
  - every FP64 value v is split into h = v truncated to 24 significant bits and
    l = the next 23 bits of v (truncated), |v - h - l| < 2^-46 |v|; values below
    2^-100 in magnitude become zero;
  - the diagonal c is split by rounding: c_h = fl32(c), c_l = fl32(c - c_h);
  - r = f + u + d + l + r' - c x (u, d the block-row neighbours, l, r' the
    in-block neighbours, all with coefficient one) is formed as: TwoSum of the
    h parts (u+d, l+r', their sum, then + f), r_hi = fl32(s - c_h x_h) in one
    rounding (FMA), lo = sum of the TwoSum errors and l parts in FP32, then
    lo -= c_h x_l, lo -= c_l x_h (FMAs), r = fl32(r_hi + lo).
FP32 additions are numpy float32 operations (IEEE, round to nearest); an FMA is
rounded once from its exact value.  The exact residual is an exactly rounded
FP64 sum (math.fsum of the terms with c x split exactly by Dekker's product).

Checked here: the stated bound |r - r_exact| <= 2^-23 |r_exact| + 2^-42 S
(S = |f| + |u| + |d| + |l| + |r'| + |c x|) on random, near-solution,
wide-magnitude and cancelling inputs; the error-free pieces (split, TwoSum,
c split); and planted mistakes that must break the bound (a dropped TwoSum
error, a dropped c_l x_h, a 12-bit low part, a plain FP32 sum).
"""

import math

import numpy as np
import pytest

import oracle
from workloads import gen

f32 = np.float32
BOUND_REL, BOUND_S = 2.0 ** -23, 2.0 ** -42


# ---------------------------------------------------------------- the method
def split(v, lo_bits=23):
    """(h, l) float32 of FP64 v: h = v truncated to 24 significant bits, l = the
    next lo_bits bits truncated; |v| < 2^-100 -> (0, 0)."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    _, e = np.frexp(a)                 # a = m 2^e, 0.5 <= m < 1
    E = e - 1                          # a in [2^E, 2^(E+1))
    h = np.floor(np.ldexp(a, 23 - E))  # 24-bit integer
    h = np.ldexp(h, E - 23)
    rest = a - h                       # exact
    l = np.ldexp(np.floor(np.ldexp(rest, 23 + lo_bits - E)), E - 23 - lo_bits)
    tiny = a < 2.0 ** -100
    h = np.where(tiny, 0.0, h)
    l = np.where(tiny, 0.0, l)
    return (np.sign(v) * h).astype(f32), (np.sign(v) * l).astype(f32)


def split_c(c):
    ch = np.asarray(c, dtype=np.float64).astype(f32)
    cl = (np.asarray(c, dtype=np.float64) - ch.astype(np.float64)).astype(f32)
    return ch, cl


def two_sum(a, b):
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def _two_sum64(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def fma32(a, b, c):
    """float32 a * b + c with one rounding (round to nearest even)."""
    a = np.asarray(a, f32).astype(np.float64)
    b = np.asarray(b, f32).astype(np.float64)
    c = np.asarray(c, f32).astype(np.float64)
    p = a * b                                  # exact: 48 significant bits
    s, e = _two_sum64(p, c)                    # p + c = s + e exactly
    r = s.astype(f32)
    # s is the FP64 rounding of p + c; rounding s to FP32 can differ from
    # rounding p + c only when s is an FP32 tie (the midpoint of two FP32
    # neighbours) and e != 0: the exact value then lies on e's side
    r64 = r.astype(np.float64)
    other = np.where(r64 > s, np.nextafter(r, f32(-np.inf)), np.nextafter(r, f32(np.inf))).astype(f32)
    o64 = other.astype(np.float64)
    tie = (r64 != s) & ((r64 + o64) * 0.5 == s) & (e != 0)
    hi = np.maximum(r, other)
    lo = np.minimum(r, other)
    r = np.where(tie & (e > 0), hi, np.where(tie & (e < 0), lo, r))
    return r.astype(f32)


def dw_residual(F, X, cdiag, drop_e=False, drop_clxh=False, lo_bits=23, plain=False):
    """The method on a [N, M, K] panel of a unit stencil with diagonal cdiag [N, M]."""
    N, M, K = X.shape
    z = np.zeros((1, M, K))
    U = np.concatenate([z, X[:-1]], 0)
    D = np.concatenate([X[1:], z], 0)
    zm = np.zeros((N, 1, K))
    Lf = np.concatenate([zm, X[:, :-1]], 1)
    Rt = np.concatenate([X[:, 1:], zm], 1)
    fh, fl = split(F, lo_bits)
    uh, ul = split(U, lo_bits)
    dh, dl = split(D, lo_bits)
    lh, ll = split(Lf, lo_bits)
    rh, rl = split(Rt, lo_bits)
    xh, xl = split(X, lo_bits)
    ch, cl = split_c(np.broadcast_to(cdiag[:, :, None], X.shape))
    if plain:
        return (fh + uh + dh + lh + rh - ch * xh).astype(f32)
    s1, e1 = two_sum(uh, dh)
    s2, e2 = two_sum(lh, rh)
    s3, e3 = two_sum(s1, s2)
    s4, e4 = two_sum(s3, fh)
    rhi = fma32(-ch, xh, s4)
    if drop_e:
        e4 = np.zeros_like(e4)
    lo = ((e1 + e2) + (e3 + e4)) + ((ul + dl) + (ll + rl)) + fl
    lo = fma32(-ch, xl, lo)
    if not drop_clxh:
        lo = fma32(-cl, xh, lo)
    return (rhi + lo).astype(f32)


# ---------------------------------------------------------------- exact residual
def _dekker(a, b):
    """a * b = p + e exactly (Veltkamp splitting, FP64, no FMA)."""
    fac = 134217729.0  # 2^27 + 1
    def sp(x):
        t = fac * x
        hi = t - (t - x)
        return hi, x - hi
    p = a * b
    ah, al = sp(a)
    bh, bl = sp(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def exact_residual(F, X, cdiag):
    N, M, K = X.shape
    out = np.empty_like(F)
    S = np.empty_like(F)
    for j in range(N):
        for m in range(M):
            c = float(cdiag[j, m])
            for n in range(K):
                x = float(X[j, m, n])
                terms = [float(F[j, m, n])]
                if j > 0:
                    terms.append(float(X[j - 1, m, n]))
                if j + 1 < N:
                    terms.append(float(X[j + 1, m, n]))
                if m > 0:
                    terms.append(float(X[j, m - 1, n]))
                if m + 1 < M:
                    terms.append(float(X[j, m + 1, n]))
                p, e = _dekker(c, x)
                out[j, m, n] = math.fsum(terms + [-p, -e])
                S[j, m, n] = math.fsum(abs(t) for t in terms) + abs(c * x)
    return out, S


def _bound_ok(r, F, X, cd, slack_abs=0.0):
    re, S = exact_residual(F, X, cd)
    err = np.abs(r.astype(np.float64) - re)
    bound = BOUND_REL * np.abs(re) + BOUND_S * S + slack_abs
    return bool(np.all(err <= bound)), float(np.max(err / (BOUND_REL * np.abs(re) + BOUND_S * S + 1e-300)))


def _acoustic(N, M, K, seed):
    A, B, C = gen.acoustic_system(N, M)
    F = gen.acoustic_rhs(N, M, K, seed=seed)
    cd = np.einsum("jmm->jm", C).copy()
    return A, B, C, F, cd


# ---------------------------------------------------------------- error-free pieces
def test_split_truncates_to_24_plus_23_bits():
    rng = np.random.default_rng(0)
    v = rng.standard_normal(20000) * np.exp2(rng.integers(-90, 90, 20000))
    h, l = split(v)
    hv, lv = h.astype(np.float64), l.astype(np.float64)
    d = v - hv - lv
    assert np.all(np.abs(d) < 2.0 ** -46 * np.abs(v))
    assert np.all(np.abs(lv) < 2.0 ** -23 * np.abs(v))
    assert np.all((np.sign(hv) == np.sign(v)) & ((lv == 0) | (np.sign(lv) == np.sign(v))))
    # h is v truncated: |h| <= |v| and v - h < one unit of h's last place
    assert np.all(np.abs(hv) <= np.abs(v))
    # below 2^-100 the split is zero
    h2, l2 = split(np.array([2.0 ** -101, -3e-31, 2.0 ** -100]))
    assert h2[0] == 0 and l2[0] == 0 and h2[1] == 0 and h2[2] != 0


def test_two_sum_is_exact_and_c_split_bound():
    rng = np.random.default_rng(1)
    a = (rng.standard_normal(50000) * np.exp2(rng.integers(-30, 30, 50000))).astype(f32)
    b = (rng.standard_normal(50000) * np.exp2(rng.integers(-30, 30, 50000))).astype(f32)
    s, e = two_sum(a, b)
    assert np.all(s.astype(np.float64) + e.astype(np.float64) == a.astype(np.float64) + b.astype(np.float64))
    c = 4.25 + rng.random(1000) * 2.0
    ch, cl = split_c(c)
    assert np.all(np.abs(c - ch.astype(np.float64) - cl.astype(np.float64)) <= 2.0 ** -48 * c)


def test_fma32_rounds_once():
    # a*b + c whose FP64 rounding lands on an FP32 tie: one rounding keeps the
    # exact value's side
    a = f32(1.0 + 2.0 ** -12)
    b = f32(1.0 + 2.0 ** -12)
    c = f32(-1.0)
    # exact: 2^-11 + 2^-24, representable in FP32
    assert fma32(a, b, c) == f32(2.0 ** -11 + 2.0 ** -24)
    x = np.array([3.0, -7.5], f32)
    assert np.all(fma32(x, x, f32(1.0)) == np.array([10.0, 57.25], f32))


# ---------------------------------------------------------------- the stated bound
def test_bound_random_values():
    N, M, K = 6, 16, 5
    _, _, _, F, cd = _acoustic(N, M, K, seed=1)
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (N, M, K))
    ok, worst = _bound_ok(dw_residual(F, X, cd), F, X, cd)
    assert ok, worst


def test_bound_near_the_solution():
    # the case the refinement lives in: r tiny against every term
    N, M, K = 8, 16, 4
    A, B, C, F, cd = _acoustic(N, M, K, seed=3)
    X = oracle.solve_block_thomas(A, B, C, F)
    rng = np.random.default_rng(4)
    for pert in (1e-6, 1e-11, 0.0):
        Xp = X * (1.0 + pert * rng.standard_normal(X.shape))
        r = dw_residual(F, Xp, cd)
        ok, worst = _bound_ok(r, F, Xp, cd)
        assert ok, (pert, worst)
    # and the error there is far below the bound (about 2^-46 S observed)
    r = dw_residual(F, X, cd)
    re, S = exact_residual(F, X, cd)
    assert np.max(np.abs(r - re) / S) < 2.0 ** -44


def test_bound_wide_magnitudes_and_cancellation():
    N, M, K = 5, 8, 6
    rng = np.random.default_rng(5)
    X = rng.standard_normal((N, M, K)) * np.exp2(rng.integers(-60, 60, (N, M, K)))
    cd = 4.0 + rng.random((N, M)) * 3.0
    # F chosen so that the exact residual nearly cancels: F = c x - neighbours (FP64)
    nb = np.zeros_like(X)
    nb[1:] += X[:-1]
    nb[:-1] += X[1:]
    nb[:, 1:] += X[:, :-1]
    nb[:, :-1] += X[:, 1:]
    F = cd[:, :, None] * X - nb
    ok, worst = _bound_ok(dw_residual(F, X, cd), F, X, cd)
    assert ok, worst


def test_tiny_values_are_zero_within_the_stated_allowance():
    N, M, K = 4, 8, 3
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, (N, M, K))
    X[1, 3, :] = 3e-31   # below 2^-100: counted as zero
    F = rng.uniform(-1, 1, (N, M, K))
    cd = np.full((N, M), 4.5)
    ok, _ = _bound_ok(dw_residual(F, X, cd), F, X, cd, slack_abs=6 * 2.0 ** -100 * 5)
    assert ok


# ---------------------------------------------------------------- planted mistakes
@pytest.mark.parametrize("mistake", ["drop_e", "drop_clxh", "lo12", "plain"])
def test_planted_mistakes_break_the_bound(mistake):
    N, M, K = 8, 16, 4
    A, B, C, F, cd = _acoustic(N, M, K, seed=7)
    X = oracle.solve_block_thomas(A, B, C, F)
    kw = {"drop_e": dict(drop_e=True), "drop_clxh": dict(drop_clxh=True), "lo12": dict(lo_bits=12),
          "plain": dict(plain=True)}[mistake]
    ok, worst = _bound_ok(dw_residual(F, X, cd, **kw), F, X, cd)
    assert not ok and worst > 4.0, worst
