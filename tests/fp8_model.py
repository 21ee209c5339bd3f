"""Stage 2 of Algorithm 2 with narrow tensor-core operands: a CPU model (test infrastructure).

The experiment: how does the FP64-residual refinement converge when the panel
contractions of stage 2 take FP8 operands?  The model runs the solve phase of
Section 2.2 exactly as the library's tensor-core path arranges it -- per segment
the forward recurrence y_i = Dinv_i r_i + E_i y_{i-1} (for A_i = I the product
Dinv_i (r_i + y_{i-1})), the backward recurrence W_i = y_i + G_i W_{i+1}
(eq. sub3), the interface right-hand side F~ of eq. red1, the reduced system, and
the superposition X_i = W_i + U_i X~_s + V_i X~_{s+1} -- with every block
product's two operands rounded to a format and the products accumulated in FP32,
inside the refinement X <- X + S~(F - P X) with the residual exact in FP64.
The reduced system is solved in FP64 (the model isolates the bulk contractions).

Formats:
  "e4m3"  FP8 E4M3 (OCP 8-bit format: 4 exponent bits, bias 7, 3 fraction bits,
          largest finite 448, subnormals down to 2^-9) with one power-of-two
          scale per 32 consecutive elements along the contraction (the MX block
          layout): scale 2^ceil(log2(amax / 448)), so no element saturates;
  "bf16"  BF16 (8 significant bits), "tf32" (11), "fp32", "fp64" (no rounding).
Products of two E4M3 values are exact in FP32, so this computes what an FP8
tensor-core MMA with FP32 accumulation computes, up to the summation order.

Run as a script it prints the study on the acoustic operator of the precision
workload (N = 4096, M = 128, S = 64, a sample of its right-hand sides).
"""

from __future__ import annotations

import os
import sys

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402

E4M3_MAX = 448.0


def round_bits(x, bits):
    """Round to nearest even keeping `bits` significant bits (unbounded exponent)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)  # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(np.ldexp(m, bits)), e - bits)


def round_e4m3(x):
    """Round to the nearest E4M3 value (ties to even); |x| must not exceed 448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, e = np.frexp(a)  # a = f 2^e, 0.5 <= f < 1: the leading bit is 2^(e-1)
    # quantum: 2^(e-1-3) for normal values (leading exponent >= -6), 2^-9 below
    q = np.ldexp(1.0, np.maximum(e - 1, -6) - 3)
    out = np.sign(x) * np.rint(a / q) * q
    return np.where(a == 0, 0.0, out)


def quant_mx(x, axis):
    """E4M3 with one power-of-two scale per 32 consecutive elements along `axis`."""
    x = np.moveaxis(np.asarray(x, dtype=np.float64), axis, -1)
    n = x.shape[-1]
    pad = (-n) % 32
    xp = np.concatenate([x, np.zeros(x.shape[:-1] + (pad,))], axis=-1) if pad else x
    blk = xp.reshape(xp.shape[:-1] + (xp.shape[-1] // 32, 32))
    amax = np.abs(blk).max(axis=-1, keepdims=True)
    s = np.where(amax > 0, np.ldexp(1.0, np.ceil(np.log2(np.where(amax > 0, amax, 1.0) / E4M3_MAX)).astype(int)),
                 1.0)
    q = round_e4m3(blk / s) * s
    q = q.reshape(xp.shape)[..., :n]
    return np.moveaxis(q, -1, axis)


def quant(x, fmt, axis):
    if fmt == "e4m3":
        return quant_mx(x, axis)
    if fmt == "bf16":
        return round_bits(x, 8)
    if fmt == "tf32":
        return round_bits(x, 11)
    if fmt == "fp32":
        return np.asarray(x, dtype=np.float32).astype(np.float64)
    return np.asarray(x, dtype=np.float64)


def _acc(x, fmt):
    # FP32 accumulation of the tensor-core formats (the FP64 reference keeps FP64)
    return x if fmt == "fp64" else x.astype(np.float32).astype(np.float64)


class Stage2Model:
    """Factors of stage 1 in FP64 (by the recurrences of eqs. sub1-sub3 and
    red1), then solve(r, fmt): stage 2 with operands rounded to `fmt`."""

    def __init__(self, A, B, C, S):
        N, M, _ = C.shape
        if N % S:
            raise ValueError("S must divide N")
        L = N // S
        self.N, self.M, self.S, self.L = N, M, S, L
        self.A, self.B, self.C = A, B, C
        eye = np.eye(M)
        self.unit = bool(np.all(A[1:] == eye) and np.all(B[:-1] == eye))
        Ag = A.reshape(S, L, M, M)
        Bg = B.reshape(S, L, M, M)
        Cg = C.reshape(S, L, M, M)
        Dinv = np.zeros((S, L, M, M))
        G = np.zeros((S, L, M, M))
        E = np.zeros((S, L, M, M))
        for i in range(1, L):  # interior rows 1..L-1 of every segment, all segments at once
            D = Cg[:, i] - (Ag[:, i] @ G[:, i - 1] if i > 1 else 0.0)
            Dinv[:, i] = np.linalg.inv(D)
            G[:, i] = Dinv[:, i] @ Bg[:, i]
            E[:, i] = Dinv[:, i] @ Ag[:, i]
        # responses: Y_1 = E_1, Y_i = E_i Y_{i-1}; U_i = Y_i + G_i U_{i+1}, V_i = G_i V_{i+1}
        Y = np.zeros_like(E)
        U = np.zeros_like(E)
        V = np.zeros_like(E)
        for i in range(1, L):
            Y[:, i] = E[:, i] if i == 1 else E[:, i] @ Y[:, i - 1]
        for i in range(L - 1, 0, -1):
            U[:, i] = Y[:, i] + (G[:, i] @ U[:, i + 1] if i < L - 1 else 0.0)
            V[:, i] = G[:, i] if i == L - 1 else G[:, i] @ V[:, i + 1]
        self.Dinv, self.G, self.E, self.U, self.V = Dinv, G, E, U, V
        # reduced system (eq. red1) on the interface rows k_s = s L:
        #   -At_s X~_{s-1} + Ct_s X~_s - Bt_s X~_{s+1} = F~_s
        At = np.zeros((S, M, M))
        Bt = np.zeros((S, M, M))
        Ct = np.array(Cg[:, 0])
        for s in range(S):
            Ak, Bk = Ag[s, 0], Bg[s, 0]
            if L > 1:  # the segment's own first interior row couples forward
                Ct[s] -= Bk @ U[s, 1]
                Bt[s] = Bk @ V[s, 1]
            if s > 0:
                if L > 1:
                    At[s] = Ak @ U[s - 1, L - 1]
                    Ct[s] -= Ak @ V[s - 1, L - 1]
                else:
                    At[s] = Ak
            if L == 1 and s < S - 1:
                Bt[s] = Bk
        self.At, self.Bt, self.Ct = At, Bt, Ct
        self.q = {}

    def _factors(self, fmt):
        if fmt not in self.q:
            f = lambda X: quant(X, fmt, axis=-1)  # noqa: E731 - contraction over the columns
            self.q[fmt] = {k: f(getattr(self, k)) for k in ("Dinv", "G", "E", "U", "V")}
            self.q[fmt]["A"] = f(self.A.reshape(self.S, self.L, self.M, self.M))
            self.q[fmt]["B"] = f(self.B.reshape(self.S, self.L, self.M, self.M))
        return self.q[fmt]

    def solve(self, F, fmt):
        """X = S~ F with `fmt` operands and FP32 accumulation ([N, M, K] FP64)."""
        S, L, M = self.S, self.L, self.M
        K = F.shape[2]
        qf = self._factors(fmt)
        P = lambda X: quant(X, fmt, axis=-2)  # noqa: E731 - panel operand: contraction over m
        acc = lambda X: _acc(X, fmt)  # noqa: E731
        Fg = F.reshape(S, L, M, K)
        r = quant(Fg, fmt, axis=-2) if fmt != "fp64" else Fg
        # forward: y_i = Dinv_i r_i + E_i y_{i-1}
        y = np.zeros((S, L, M, K))
        for i in range(1, L):
            if self.unit:
                t = r[:, i] + (y[:, i - 1] if i > 1 else 0.0)
                y[:, i] = acc(qf["Dinv"][:, i] @ P(acc(t)))
            else:
                v = qf["Dinv"][:, i] @ P(r[:, i])
                if i > 1:
                    v = v + qf["E"][:, i] @ P(y[:, i - 1])
                y[:, i] = acc(v)
        # backward: W_i = y_i + G_i W_{i+1}
        W = np.zeros_like(y)
        for i in range(L - 1, 0, -1):
            W[:, i] = y[:, i] if i == L - 1 else acc(y[:, i] + qf["G"][:, i] @ P(W[:, i + 1]))
        # interface right-hand side and the reduced solve (FP64)
        Ft = np.array(Fg[:, 0])
        for s in range(S):
            if L > 1:
                Ft[s] += (qf["B"][s, 0] @ P(W[s, 1])) if not self.unit else W[s, 1]
            if s > 0 and L > 1:
                Ft[s] += (qf["A"][s, 0] @ P(W[s - 1, L - 1])) if not self.unit else W[s - 1, L - 1]
        Xt = oracle.solve_block_thomas(self.At, self.Bt, self.Ct, acc(Ft))
        # superposition: X_i = W_i + U_i X~_s + V_i X~_{s+1}
        X = np.zeros_like(y)
        X[:, 0] = Xt
        Xn = np.concatenate([Xt[1:], np.zeros((1, M, K))], axis=0)
        for i in range(1, L):
            X[:, i] = acc(W[:, i] + qf["U"][:, i] @ P(Xt) + qf["V"][:, i] @ P(Xn))
        return X.reshape(self.N, M, K)


def refine(model, F, fmt, tol=1e-10, max_it=40):
    """The FP64-residual refinement; returns (X, [||F - P X_k|| / ||F|| for k = 0, 1, ...])."""
    A, B, C = model.A, model.B, model.C
    fn = np.linalg.norm(F)
    X = model.solve(F, fmt)
    hist = [np.linalg.norm(oracle.residual(A, B, C, X, F)) / fn]
    while hist[-1] > tol and len(hist) <= max_it:
        R = oracle.residual(A, B, C, X, F)
        X = X + model.solve(R, fmt)
        hist.append(np.linalg.norm(oracle.residual(A, B, C, X, F)) / fn)
    return X, hist


def study(N=4096, M=128, S=64, K=16, seed=0, formats=("e4m3", "bf16", "tf32"), tol=1e-10):
    from workloads import gen

    A, B, C = gen.acoustic_system(N, M)
    F = gen.acoustic_rhs(N, M, 512, seed=seed)
    F = np.ascontiguousarray(F[:, :, np.linspace(0, 511, K).round().astype(int)])
    model = Stage2Model(A, B, C, S)
    out = {}
    for fmt in formats:
        _, hist = refine(model, F, fmt, tol=tol)
        out[fmt] = hist
    return out


if __name__ == "__main__":
    res = study()
    for fmt, hist in res.items():
        red = [hist[k + 1] / hist[k] for k in range(len(hist) - 1)]
        print(f"{fmt}: passes after the first solve {len(hist) - 1}; rel. residual per solve "
              + " ".join(f"{h:.2e}" for h in hist)
              + ("; reduction per pass " + " ".join(f"{v:.2e}" for v in red) if red else ""))
