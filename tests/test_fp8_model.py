"""Pins of the narrow-operand stage-2 model (tests/fp8_model.py).

CPU: the E4M3 rounding against every code of the format, decoded from its bit
fields; the MX block quantiser's scale and error; BF16 rounding against
torch's; the model without rounding reproduces the oracle's block-Thomas
solution on unit-stencil and dense systems with S = 1, several segments and
S = N (a dropped response term, a transposed factor or a wrong interface
coupling fails these); a planted error in the model is caught.
GPU: the model's BF16 and TF32 first-solve residuals agree with the library's
tensor-core solves of the same panels (the model captures their numerics).
"""

import numpy as np
import pytest

import oracle
from workloads import gen

import fp8_model as fm


def _e4m3_table():
    """Every finite E4M3 value from its bit fields (sign, 4-bit exponent with
    bias 7, 3-bit fraction; exponent 0 subnormal; S.1111.111 is NaN)."""
    vals = []
    for code in range(256):
        s, e, m = code >> 7, (code >> 3) & 15, code & 7
        if e == 15 and m == 7:
            continue
        mag = 2.0 ** -6 * (m / 8) if e == 0 else 2.0 ** (e - 7) * (1 + m / 8)
        vals.append(((-1) ** s * mag, m))
    return vals


def test_e4m3_rounding_matches_the_format():
    table = _e4m3_table()
    v = np.array([t[0] for t in table])
    assert np.max(v) == 448.0 and np.min(np.abs(v[v != 0])) == 2.0 ** -9
    assert np.array_equal(fm.round_e4m3(v), v)  # representable values stay
    pos = np.unique(v[v >= 0])
    mant = {val: m for val, m in table if val >= 0}
    mids = (pos[:-1] + pos[1:]) / 2
    got = fm.round_e4m3(mids)
    for lo, hi, g in zip(pos[:-1], pos[1:], got):  # ties go to the even fraction
        assert g == (lo if mant[lo] % 2 == 0 else hi), (lo, hi, g)
    rng = np.random.default_rng(1)
    x = rng.uniform(-448, 448, 4000) * np.exp2(rng.integers(-12, 0, 4000))
    near = pos[np.argmin(np.abs(np.abs(x)[:, None] - pos[None, :]), axis=1)] * np.sign(x)
    assert np.array_equal(np.abs(fm.round_e4m3(x) - x), np.abs(near - x))


def test_mx_blocks():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 70, 5)) * np.exp2(rng.integers(-30, 30, (3, 1, 5)))
    q = fm.quant_mx(x, axis=1)
    grid = set(t[0] for t in _e4m3_table())
    for b in range(3):
        for c in range(5):
            for j0 in range(0, 70, 32):
                blk, qb = x[b, j0:j0 + 32, c], q[b, j0:j0 + 32, c]
                s = 2.0 ** np.ceil(np.log2(np.abs(blk).max() / 448.0))
                assert all((v / s) in grid for v in qb)
                assert 224.0 < np.abs(blk).max() / s <= 448.0
                normal = np.abs(blk) >= 2.0 ** -6 * s
                assert np.all(np.abs(qb - blk)[normal] <= 2.0 ** -4 * np.abs(blk)[normal])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(3).standard_normal(5000).astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(fm.round_bits(x, 8), ref)


@pytest.mark.parametrize("kind,N,M,S", [("acoustic", 48, 16, 4), ("acoustic", 16, 8, 16), ("acoustic", 24, 8, 1),
                                        ("dense", 40, 6, 5), ("dense", 12, 4, 12), ("dense", 30, 5, 1)])
def test_model_without_rounding_is_the_solve(kind, N, M, S):
    if kind == "acoustic":
        A, B, C = gen.acoustic_system(N, M)
    else:
        A, B, C = gen.dominant_blocks(N, M, seed=N)
    F = gen.uniform_rhs(N, M, 3, seed=7)
    X = fm.Stage2Model(A, B, C, S).solve(F, "fp64")
    assert oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-12


def test_a_planted_error_in_the_model_is_caught():
    A, B, C = gen.dominant_blocks(40, 6, seed=40)
    F = gen.uniform_rhs(40, 6, 3, seed=7)
    m = fm.Stage2Model(A, B, C, 5)
    m.V = np.swapaxes(m.V, -1, -2).copy()  # a transposed coupling response
    assert oracle.rel_err(m.solve(F, "fp64"), oracle.solve_block_thomas(A, B, C, F)) > 1e-6


def test_refinement_converges_with_narrow_operands():
    A, B, C = gen.acoustic_system(64, 32)
    F = gen.acoustic_rhs(64, 32, 4, seed=1)
    m = fm.Stage2Model(A, B, C, 8)
    for fmt in ("bf16", "e4m3"):
        X, hist = fm.refine(m, F, fmt, tol=1e-12)
        assert hist[-1] <= 1e-12 and oracle.rel_err(X, oracle.solve_block_thomas(A, B, C, F)) <= 1e-10
    # narrower operands reduce the residual less per solve
    _, hb = fm.refine(m, F, "bf16", tol=1e-12)
    _, h8 = fm.refine(m, F, "e4m3", tol=1e-12)
    assert h8[0] > 4 * hb[0] and len(h8) >= len(hb)


@pytest.mark.gpu
@pytest.mark.parametrize("fmt", ["bf16", "tf32"])
def test_model_matches_the_tensor_core_solve(fmt):
    torch = pytest.importorskip("torch")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1108_4181_gb300 as bt

    N, M, K, S = 512, 128, 16, 16
    A, B, C = gen.acoustic_system(N, M)
    F = gen.acoustic_rhs(N, M, K, seed=3)
    model0 = fm.Stage2Model(A, B, C, S).solve(F, fmt)
    r_model = np.linalg.norm(oracle.residual(A, B, C, model0, F)) / np.linalg.norm(F)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")  # noqa: E731
    with bt.factor(t(A), t(B), t(C), S) as fac:
        _, info = fac.solve(t(F), precision=fmt, tol=1.0, return_info=True)
    assert info["iters"] == 0
    ratio = info["rel_res0"] / r_model
    assert 0.25 <= ratio <= 4.0, (info["rel_res0"], r_model)
