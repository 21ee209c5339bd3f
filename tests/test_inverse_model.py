"""Pins of the pivot-block inversion method (the factorisation's cluster kernel) on the CPU.

The kernel runs Gauss-Jordan with partial pivoting with the row scaling
deferred: the rows keep their raw values U, row k records s_k = 1 / pivot, and
step k (after interchanging rows k and p) is

    g_i = U[i][k] / pivot,   U[i][j] -= g_i U[k][j]  (i != k, j != k),
    U[i][k] = -g_i  (i != k),   U[k][k] = 1,

the textbook step applied to diag(s) U; the inverse is diag(s) U with the
interchanges undone as column interchanges.  1 / pivot is an FP32 reciprocal of
the pivot's leading significand bits (exponent from the bits) refined by two
Newton-Raphson steps.  Here the method is written out in numpy, in the
kernel's order, and held against LAPACK's inverse and against the textbook
Gauss-Jordan with immediate scaling; planted mistakes (one Newton step, a
dropped deferred scale, a sign slip in the pivot column, pivots not
interchanged back) must fail.
"""

import math

import numpy as np
import pytest


def recip_newton(v, steps=2):
    """1 / v: FP32 reciprocal of the leading 23 significand bits, then Newton-Raphson."""
    m, e = math.frexp(abs(v))                      # |v| = m 2^e, m in [0.5, 1)
    m2 = np.float32(np.floor(m * 2.0 ** 24) / 2.0 ** 23)  # 1.f truncated to 23 bits, in [1, 2)
    r = float(np.float32(1.0) / m2) * 2.0 ** (1 - e)
    r = math.copysign(r, v)
    for _ in range(steps):
        r = r + r * (1.0 - v * r)
    return r


def gj_deferred(A, newton_steps=2, drop_scale=False, sign_slip=False, undo=True):
    """The kernel's Gauss-Jordan inverse in its order of operations."""
    n = A.shape[0]
    U = np.array(A, dtype=np.float64)
    s = np.zeros(n)
    perm = np.zeros(n, dtype=int)
    for k in range(n):
        col = np.abs(U[k:, k])
        p = k + int(np.argmax(col))                # the first of equal maxima: the lower row
        perm[k] = p
        if p != k:
            U[[k, p]] = U[[p, k]]
        rinv = recip_newton(U[k, k], newton_steps)
        g = U[:, k] * rinv
        pivot_row = U[k].copy()
        for i in range(n):
            if i == k:
                continue
            U[i] -= g[i] * pivot_row
            U[i, k] = g[i] if sign_slip else -g[i]
        U[k, k] = 1.0
        s[k] = 1.0 if drop_scale else rinv
    X = s[:, None] * U
    if undo:  # the row interchanges, undone as column interchanges in reverse order
        for k in range(n - 1, -1, -1):
            p = perm[k]
            if p != k:
                X[:, [k, p]] = X[:, [p, k]]
    return X


def gj_textbook(A):
    """Gauss-Jordan with partial pivoting and immediate row scaling."""
    n = A.shape[0]
    T = np.array(A, dtype=np.float64)
    perm = []
    for k in range(n):
        p = k + int(np.argmax(np.abs(T[k:, k])))
        perm.append(p)
        T[[k, p]] = T[[p, k]]
        pv = T[k, k]
        T[k] /= pv
        T[k, k] = 1.0 / pv
        for i in range(n):
            if i != k:
                f = T[i, k]
                T[i] -= f * T[k]
                T[i, k] = -f / pv
    for k in range(n - 1, -1, -1):
        p = perm[k]
        T[:, [k, p]] = T[:, [p, k]]
    return T


def _matrices():
    rng = np.random.default_rng(3)
    n = 24
    dom = rng.random((n, n)) - 0.5
    dom[np.arange(n), np.arange(n)] = np.abs(dom).sum(1) + 1.0
    gen = rng.standard_normal((n, n))                      # general: pivoting interchanges rows
    scaled = gen * np.exp2(rng.integers(-300, 300, (1, n)))  # columns over 2^-300..2^300
    return {"dominant": dom, "general": gen, "scaled_columns": scaled}


def test_recip_newton_is_accurate_over_the_exponent_range():
    rng = np.random.default_rng(1)
    vals = rng.uniform(1.0, 2.0, 3000) * np.exp2(rng.integers(-1000, 1000, 3000)) * rng.choice([-1.0, 1.0], 3000)
    for v in vals:
        r = recip_newton(float(v))
        assert abs(r * v - 1.0) <= 2.0 ** -51, v
    # one Newton step from the 23-bit seed stops near 2^-48
    worst = max(abs(recip_newton(float(v), 1) * v - 1.0) for v in vals)
    assert worst > 2.0 ** -51


@pytest.mark.parametrize("name", ["dominant", "general", "scaled_columns"])
def test_deferred_scaling_inverse_matches_lapack_and_textbook(name):
    A = _matrices()[name]
    X = gj_deferred(A)
    Xl = np.linalg.inv(A)
    Xt = gj_textbook(A)
    # column scaling of A scales the rows of the inverse: compare row by row
    rs = np.abs(Xl).max(axis=1, keepdims=True)
    assert np.max(np.abs(X - Xl) / rs) <= 1e-13
    assert np.max(np.abs(X - Xt) / rs) <= 1e-13
    # the residual in the scale-free form |A X - I|
    assert np.max(np.abs(A @ X - np.eye(A.shape[0]))) <= 1e-12


def test_planted_mistakes_fail():
    A = _matrices()["general"]
    Xl = np.linalg.inv(A)
    rs = np.abs(Xl).max(axis=1, keepdims=True)

    def err(**kw):
        return np.max(np.abs(gj_deferred(A, **kw) - Xl) / rs)

    assert err() <= 1e-13
    assert err(newton_steps=1) > 4 * err()  # one Newton step leaves ~2^-48 in every row scale
    assert err(drop_scale=True) > 1e-3      # the deferred row scales forgotten
    assert err(sign_slip=True) > 1e-3       # column k of the inverse with the wrong sign
    assert err(undo=False) > 1e-3           # interchanges not undone
