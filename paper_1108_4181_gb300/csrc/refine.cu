// Mixed-precision solve with iterative refinement (not in the paper).
//
//   X_0 = S~ F,   X_{k+1} = X_k + S~ (F - P X_k)
//
// S~ is Algorithm 2's stage 2 run with rounded factors (FP32 on the CUDA cores,
// or BF16 / TF32 on the tensor cores with FP32 accumulation); the residual
// F - P X is formed in FP64 from the operator kept in the handle.  The loop is
// unrolled on the host with a device-side stop flag: after every residual a
// one-thread kernel compares ||r||_F^2 with tol^2 ||F||_F^2, and once the flag
// is set every later kernel of the sequence returns at once, so the whole
// refinement is enqueued without a host round trip.

#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include "bt_internal.cuh"
#include "fpconv.cuh"

namespace bt {

namespace {

constexpr int kMaxPasses = 64;

struct IrState {
  double fn2;               // ||F||_F^2
  double rn2[kMaxPasses];   // ||F - P X_k||_F^2
  int done;                 // 1 converged, 2 stalled
  int last;                 // index of the last residual computed
  int solves;               // refinement solves performed after the first
  int kstatus;              // non-zero: a tensor-core kernel gave up a bounded wait
  int cur;                  // slot of the next residual (advanced by every check)
  int range;                // the FP32 double-word residual met a value it cannot represent
  double rn2_fb;            // ||r||_F^2 of the FP64 residual that then replaced it
  int setok;                // per-set criterion (k_set_check): every column set within tolerance
};

template <typename T>
__device__ __forceinline__ T to_lp(double v);
template <>
__device__ __forceinline__ float to_lp<float>(double v) { return f64_to_f32_rz(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_lp<__nv_bfloat16>(double v) { return __double2bfloat16(v); }
template <>
__device__ __forceinline__ double to_lp<double>(double v) { return v; }
__device__ __forceinline__ float lp_to_float(float v) { return v; }
__device__ __forceinline__ float lp_to_float(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ void block_add(double v, double* target) {
  __shared__ double red[32];
  __syncthreads();  // red[] may still be read by a previous call
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < (int)(blockDim.x / 32) ? red[l] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (l == 0 && v != 0.0) atomicAdd(target, v);
  }
}

// Sum of squares of FP32 values with a per-thread power-of-two scale: a value
// v enters as (v 2^-e)^2; when one of magnitude 2^(e+32) or more arrives, e
// is raised to its exponent and the sum rescaled, so the squares neither
// overflow (|v| up to FP32's largest) nor lose the values near the largest
// one; values below 2^(e-74) vanish, at most 2^-148 of the largest square
// each.  total() is the sum in FP64.
struct Ssq {
  float acc = 0.f;
  float f = 0x1p100f;   // 2^-e
  float thr = 0x1p-68f; // 2^(e+32); +inf once e + 32 > 127
  int e = -100;
  __device__ __forceinline__ void add(float v) {
    if (fabsf(v) >= thr) rescale(v);
    const float w = v * f;
    acc = fmaf(w, w, acc);
  }
  __device__ __forceinline__ void rescale(float v) {
    const int ev = (int)((__float_as_uint(v) >> 23) & 0xffu) - 127;
    const int en = min(ev, 126);
    const int d = 2 * (e - en);  // <= -64
    acc *= d >= -126 ? __int_as_float((127 + d) << 23) : 0.f;
    e = en;
    f = __int_as_float((127 - en) << 23);
    thr = en + 32 <= 127 ? __int_as_float((127 + en + 32) << 23) : __int_as_float(0x7f800000);
  }
  __device__ __forceinline__ double total() const {
    return (double)acc * __hiloint2double((1023 + 2 * e) << 20, 0);
  }
};

// One residual entry of the stencil operator (A_j = B_j = I, tridiagonal C_j):
// r = F_j + X_{j-1} + X_{j+1} - C_j X_j at (j, m, n), FP64.
__device__ __forceinline__ double stencil_res(const double* __restrict__ F, const double* __restrict__ X,
                                              const double* __restrict__ Cd, int64_t N, int M, int64_t K, int64_t j,
                                              int m, int64_t n, int first) {
  // FP64 instructions are the scarce resource on this GPU (about 1/60 of the
  // FP32 rate): five fused operations per entry, no separate products.
  const size_t MK = (size_t)M * K;
  const size_t e = j * MK + (size_t)m * K + n;
  double v = F[e];
  if (!first) {
    const double* cd = Cd + 3 * (j * M + m);
    v = fma(-cd[1], X[e], v);
    if (m > 0) v = fma(-cd[0], X[e - K], v);
    if (m + 1 < M) v = fma(-cd[2], X[e + K], v);
    if (j > 0) v += X[e - MK];
    if (j + 1 < N) v += X[e + MK];
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Stores v at r[idx]; with two planes (sp = 2) the rounded value goes to plane 0
// and the rounding remainder to plane 1 (r[idx + plane]).
__device__ __forceinline__ void put_planes(__nv_bfloat16* r, size_t idx, size_t plane, int sp, float v) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  r[idx] = hi;
  if (sp == 2) r[idx + plane] = __float2bfloat16_rn(v - __bfloat162float(hi));
}
__device__ __forceinline__ void put_planes(double* r, size_t idx, size_t, int, float v) { r[idx] = v; }
__device__ __forceinline__ void put_planes(float* r, size_t idx, size_t plane, int sp, float v) {
  if (sp == 2) {
    const float hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
    r[idx] = hi;
    r[idx + plane] = v - hi;
  } else {
    r[idx] = v;
  }
}

// Row-major residual panel (leading dimension K): grid-stride over entries.
// With `gate` non-NULL the kernel runs only when *gate is set (the fallback of
// the double-word residual) and adds its squared norm to st->rn2_fb.
template <typename TR>
__global__ void __launch_bounds__(256) k_resid_stencil(const double* __restrict__ F, const double* __restrict__ X,
                                                      const double* __restrict__ Cd, TR* __restrict__ r,
                                                      int64_t N, int M, int64_t K, int first, int pass,
                                                      IrState* st, const int* gate) {
  if (st->done || (gate != nullptr && *(volatile const int*)gate == 0)) return;
  const size_t MK = (size_t)M * K, n = (size_t)N * MK;
  double acc = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t j = e / MK;
    const size_t rem = e % MK;
    const double v = stencil_res(F, X, Cd, N, M, K, j, (int)(rem / K), rem % K, first);
    r[e] = to_lp<TR>(v);
    acc += v * v;
  }
  (void)pass;
  block_add(acc, first ? &st->fn2 : gate ? &st->rn2_fb : &st->rn2[st->cur]);
  if (first) block_add(acc, &st->rn2[0]);
}

// Block-transposed residual panel, one warp per (block row j, 8 rows m,
// 32 columns n) item: lane n loads rows m0-1 .. m0+8 of its column (every load
// a coalesced 256-byte row), so the m-neighbours of its 8 entries are in its
// own registers and its 8 results are contiguous in the block-transposed
// panel -- one 16-byte store per plane, no shared memory, no CTA barrier.
// Five FP64 operations per entry (none with X = 0); FP32 rounding and the
// squared norm off the FP64 pipe.  Requires M % 8 == 0.
template <typename TR>
__global__ void __launch_bounds__(256, 2) k_resid_warp(const double* __restrict__ F, const double* __restrict__ X,
                                                      const double* __restrict__ Cd, TR* __restrict__ r, int64_t N,
                                                      int M, int Mr, int64_t K, int64_t Kp, int pass, int sp,
                                                      IrState* st, const int* gate) {
  // Mr: rows per block row of the panel (M padded to the tensor-core tile;
  // rows past M are written as zeros)
  constexpr int first = 0;
  if (st->done || (gate != nullptr && *(volatile const int*)gate == 0)) return;
  const size_t plane = (size_t)N * Kp * Mr;
  const size_t MK = (size_t)M * K;
  const int lane = threadIdx.x % 32;
  const int tn = (int)((Kp + 31) / 32), tm = Mr / 8;
  const int64_t nitem = N * tm * tn;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  Ssq acc;
  for (int64_t it = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; it < nitem; it += warps) {
    const int n = (int)(it % tn) * 32 + lane;
    const int m0 = (int)((it / tn) % tm) * 8;
    const int64_t j = it / ((int64_t)tn * tm);
    const bool ncol = n < K;
    const double* xj = X + (size_t)j * MK + n;
    const double* fj = F + (size_t)j * MK + n;
    double f[8], xs[10], xu[8], xd[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) f[q] = (ncol && m0 + q < M) ? fj[(size_t)(m0 + q) * K] : 0.0;
    if (!first) {
#pragma unroll
      for (int q = 0; q < 10; ++q) {
        const int m = m0 - 1 + q;
        xs[q] = (ncol && m >= 0 && m < M) ? xj[(size_t)m * K] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const bool in = ncol && m0 + q < M;
        xu[q] = (in && j > 0) ? xj[(size_t)(m0 + q) * K - MK] : 0.0;
        xd[q] = (in && j + 1 < N) ? xj[(size_t)(m0 + q) * K + MK] : 0.0;
      }
    }
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int m = m0 + q;
      double w = f[q];
      if (!first && m < M) {
        const double* cd = Cd + 3 * ((size_t)j * M + m);
        w = (w + xu[q]) + xd[q];
        w = fma(-cd[1], xs[q + 1], w);
        if (m > 0) w = fma(-cd[0], xs[q], w);
        if (m + 1 < M) w = fma(-cd[2], xs[q + 2], w);
      }
      v[q] = (ncol && m < M) ? f64_to_f32_rz(w) : 0.f;
      acc.add(v[q]);
    }
    if (n < Kp) {
      TR* o = r + ((size_t)j * Kp + n) * Mr + m0;
      if constexpr (sizeof(TR) == 2) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
          const float2 bf = __bfloat1622float2(b);
          const __nv_bfloat162 c = __floats2bfloat162_rn(v[2 * q] - bf.x, v[2 * q + 1] - bf.y);
          h[q] = *reinterpret_cast<const uint32_t*>(&b);
          l[q] = *reinterpret_cast<const uint32_t*>(&c);
        }
        *reinterpret_cast<uint4*>(o) = make_uint4(h[0], h[1], h[2], h[3]);
        if (sp == 2) *reinterpret_cast<uint4*>(o + plane) = make_uint4(l[0], l[1], l[2], l[3]);
      } else {
        float hi[8], lo[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          hi[q] = sp == 2 ? __uint_as_float(__float_as_uint(v[q]) & 0xFFFFE000u) : v[q];
          lo[q] = v[q] - hi[q];
        }
        reinterpret_cast<float4*>(o)[0] = make_float4(hi[0], hi[1], hi[2], hi[3]);
        reinterpret_cast<float4*>(o)[1] = make_float4(hi[4], hi[5], hi[6], hi[7]);
        if (sp == 2) {
          reinterpret_cast<float4*>(o + plane)[0] = make_float4(lo[0], lo[1], lo[2], lo[3]);
          reinterpret_cast<float4*>(o + plane)[1] = make_float4(lo[4], lo[5], lo[6], lo[7]);
        }
      }
    }
  }
  (void)pass;
  block_add(acc.total(), first ? &st->fn2 : gate ? &st->rn2_fb : &st->rn2[st->cur]);
  if (first) block_add(acc.total(), &st->rn2[0]);
}

// ----------------------------------------------------------------------------
// The stencil residual in FP32 double-word arithmetic (not in the paper).
//
// For A_j = B_j = I and C_j = tridiag(-1, c, -1) (the unit-stencil operators)
//   r = f + x_{j-1} + x_{j+1} + x_{m-1} + x_{m+1} - c x
// per entry, where the FP64 pipe of this GPU (1/64 of the FP32 rate) would
// bound five FP64 operations per entry well below the HBM rate.  Every FP64
// value v is split on the integer pipe into two FP32 terms (dw_split): h = v
// truncated to 24 significant bits and l = the next 23 bits, so that
// |v - h - l| < 2^-46 |v|; c comes split from the factorisation (Cdw).  The
// five unit terms are summed exactly by Knuth's TwoSum on the h parts
// (errors e_1..e_4 kept), the product c x enters through one FMA whose exact
// intermediate absorbs the cancellation, r_hi = fma(-c_h, x_h, s), and every
// low-order term -- l parts, TwoSum errors, c_h x_l, c_l x_h -- is summed in
// FP32 into r = r_hi + lo.  Error per entry, against the exact residual:
//   |r - r_exact| <= 2^-23 |r_exact| + 2^-42 S,   S = |f| + |P||x| summed
// over the six terms (split truncation 2^-46 per term, dropped c_l x_l
// 2^-47, the rounding of r_hi and of the low-order sum at most 66 2^-48 S in
// all, the FP32 result 2^-23 |r|).  Values below 2^-100 in magnitude count as
// zero (an absolute error below 2^-100 each).  A value of 2^77 or more (or
// non-finite) in a warp's item sets *range; the FP64 kernel then recomputes
// the whole residual (it runs gated on that flag) and k_ir_check takes its
// norm.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// v = h + l + d with |d| < 2^-46 |v|; h, l carry v's sign.  amax collects the
// largest |v| bit pattern (high word shifted left once, sign dropped) for the
// caller's range check.
__device__ __forceinline__ void dw_split(double v, float& h, float& l, uint32_t& amax) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const uint32_t mag2 = hi << 1;
  amax = max(amax, mag2);
  // the FP64 exponent re-biased to FP32 (hi - 896 << 20 keeps the sign bit
  // for biased exponents 897..1151), shifted into place with the top 23
  // fraction bits; the shift drops the sign, which is put back
  const uint32_t hs = __funnelshift_l(lo, hi - (896u << 20), 3) | (hi & 0x80000000u);
  // eb = +-2^(E-23), one unit in the last place of h; the next 23 fraction
  // bits of v below that unit are read off as (eb with those bits) - eb, exactly
  const uint32_t eb = (hs & 0xff800000u) - (23u << 23);
  const uint32_t tb = ((lo >> 6) & 0x007fffffu) | eb;
  const bool tiny = mag2 < (923u << 21);  // |v| < 2^-100
  h = tiny ? 0.f : __uint_as_float(hs);
  l = tiny ? 0.f : __uint_as_float(tb) - __uint_as_float(eb);
}

// One entry: f + u + d + l + r - c x from double-word terms.
__device__ __forceinline__ float dw_entry(float fh, float fl, float uh, float ul, float dh, float dl, float lh,
                                          float ll, float rh, float rl, float xh, float xl, float ch, float cl) {
  float s1, e1, s2, e2, s3, e3, s4, e4;
  two_sum(uh, dh, s1, e1);
  two_sum(lh, rh, s2, e2);
  two_sum(s1, s2, s3, e3);
  two_sum(s3, fh, s4, e4);
  const float rhi = fmaf(-ch, xh, s4);  // exact intermediate, one rounding
  float lo = ((e1 + e2) + (e3 + e4)) + ((ul + dl) + (ll + rl)) + fl;
  lo = fmaf(-ch, xl, lo);
  lo = fmaf(-cl, xh, lo);
  return rhi + lo;
}

__device__ __forceinline__ uint32_t bf2_u32(__nv_bfloat162 b) { return *reinterpret_cast<const uint32_t*>(&b); }

// Rows m0 - 1 .. m0 + MC of one column of one block row of X (the item's rows
// and their halo in the block's row direction), split into double words.
template <int MC>
struct Slot {
  float h[MC + 2], l[MC + 2];
};

// One warp per item (JC block rows j, MC rows m, 32 columns n): lane n marches
// down the item's block rows keeping X_{j-1}, X_j and X_{j+1} (rows m0 - 1 ..
// m0 + MC each) split into double-word registers, so every X value is loaded
// and split once per item and its halo; the march is unrolled by three so the
// window rotates by renaming.  The next block row's X_{j+2} and F_{j+1} are
// loaded at the start of a step and split at its end.  Measured on the
// acoustic workload (N = 4096, M = 128, K = 512): 1.32 ms per residual, 0.60
// of the HBM copy rate, bound by load latency at 16 warps per SM (128
// registers; 80 registers spill and run 2.5x slower, rows fed through a TMA
// ring of small boxes or an L2 bulk prefetch ran slower).  Output: TRANS -- the
// block-transposed panel of the tensor-core solve (element (m, n) of block
// row j at (j ldr + n) M + m, ldr = Kp, columns K..Kp-1 written as zero; with
// sp = 2 the rounding remainder in plane 1); otherwise the row-major panel
// (ld = K) in FP32 or FP64.
//
// Where X comes from (SRC):
//   0  the row-major FP64 solution X, split on the integer pipe;
//   1  X = d1, a row-major [N][M][K] FP32 panel (the first solve's result,
//      exact in FP32: no split);
//   2  X = d1 + d, two such panels (the first refinement pass: the two
//      solves' results), summed exactly by TwoSum; the kernel also writes
//      X = d1 + d (FP64, exact) into the row-major solution for its own rows,
//      so the update and the residual are one pass over the panels.
// SRC 1 and 2 are used with TRANS (the tensor-core solve's residual panel).
template <typename TR, bool TRANS, int SRC>
struct DwResid {
  static constexpr int MC = 4, JC = 48;
  const double* __restrict__ F;
  const double* __restrict__ X;
  const float* __restrict__ D1;
  const float* __restrict__ D2;
  double* __restrict__ Xout;
  const float2* __restrict__ Cdw;
  TR* __restrict__ r;
  int N, K, ldr, M, sp;
  size_t plane;
  // per item
  int n, j1, m0;
  bool colok, okl, okr;
  uint32_t amax = 0;
  bool fbig = false;  // an FP32 input of magnitude 2^77 or more
  Ssq acc;

  // raw X values of one row window (FP64 for SRC 0, FP32 panel values otherwise)
  struct Raw {
    double x[SRC == 0 ? MC + 2 : 1];
    float a[SRC == 0 ? 1 : MC + 2];
    float b[SRC == 2 ? MC + 2 : 1];
  };

  __device__ __forceinline__ void load_panel(const float* __restrict__ P, bool jok, int j, float (&t)[MC + 2]) const {
    const float* p = P + ((size_t)j * M + m0 - 1) * K + n;
    t[0] = (jok && okl) ? __ldg(p) : 0.f;
#pragma unroll
    for (int q = 1; q <= MC; ++q) t[q] = (jok && colok) ? __ldg(p + (size_t)q * K) : 0.f;
    t[MC + 1] = (jok && okr) ? __ldg(p + (size_t)(MC + 1) * K) : 0.f;
  }
  __device__ __forceinline__ void load_x(int j, Raw& t) const {
    const bool jok = j >= 0 && j < N;
    if constexpr (SRC == 0) {
      const double* p = X + ((size_t)j * M + m0 - 1) * K + n;
      t.x[0] = (jok && okl) ? __ldg(p) : 0.0;
#pragma unroll
      for (int q = 1; q <= MC; ++q) t.x[q] = (jok && colok) ? __ldg(p + (size_t)q * K) : 0.0;
      t.x[MC + 1] = (jok && okr) ? __ldg(p + (size_t)(MC + 1) * K) : 0.0;
    } else {
      load_panel(D1, jok, j, t.a);
      if constexpr (SRC == 2) load_panel(D2, jok, j, t.b);
    }
  }
  __device__ __forceinline__ void load_f(int j, double (&t)[MC]) const {
    const bool jok = j >= 0 && j < N && colok;
    const double* p = F + ((size_t)j * M + m0) * K + n;
#pragma unroll
    for (int q = 0; q < MC; ++q) t[q] = jok ? __ldg(p + (size_t)q * K) : 0.0;
  }
  __device__ __forceinline__ void split_x(const Raw& t, Slot<MC>& o) {
#pragma unroll
    for (int q = 0; q < MC + 2; ++q) {
      if constexpr (SRC == 0) {
        dw_split(t.x[q], o.h[q], o.l[q], amax);
      } else if constexpr (SRC == 1) {
        o.h[q] = t.a[q];
        o.l[q] = 0.f;
        fbig = fbig || !(fabsf(t.a[q]) < 0x1p77f);
      } else {
        two_sum(t.a[q], t.b[q], o.h[q], o.l[q]);
        fbig = fbig || !(fabsf(t.a[q]) < 0x1p77f) || !(fabsf(t.b[q]) < 0x1p77f);
      }
    }
  }
  __device__ __forceinline__ void split_f(const double (&t)[MC], float (&fh)[MC], float (&fl)[MC]) {
#pragma unroll
    for (int q = 0; q < MC; ++q) dw_split(t[q], fh[q], fl[q], amax);
  }

  // Row j from U = X_{j-1}, C = X_j, D = X_{j+1}; then U <- X_{j+2}, f <- F_{j+1}.
  __device__ __forceinline__ void step(Slot<MC>& U, const Slot<MC>& C, const Slot<MC>& D, float (&fh)[MC],
                                       float (&fl)[MC], int j) {
    const bool more = j + 1 < j1;
    Raw px;
    double pf[MC];
    load_x(more ? j + 2 : -1, px);
    load_f(more ? j + 1 : -1, pf);
    const float4* cp = reinterpret_cast<const float4*>(Cdw + (size_t)j * M + m0);
    const float4 c01 = __ldg(cp), c23 = __ldg(cp + 1);
    const float ch[MC] = {c01.x, c01.z, c23.x, c23.z}, cl[MC] = {c01.y, c01.w, c23.y, c23.w};
    float v[MC];
#pragma unroll
    for (int q = 0; q < MC; ++q) {
      v[q] = dw_entry(fh[q], fl[q], U.h[q + 1], U.l[q + 1], D.h[q + 1], D.l[q + 1], C.h[q], C.l[q], C.h[q + 2],
                      C.l[q + 2], C.h[q + 1], C.l[q + 1], ch[q], cl[q]);
      acc.add(v[q]);
    }
    store(v, j);
    if constexpr (SRC == 2) {
      if (colok) {  // X = d1 + d for the item's rows of block row j (exact in FP64)
        double* o = Xout + ((size_t)j * M + m0) * K + n;
#pragma unroll
        for (int q = 0; q < MC; ++q) o[(size_t)q * K] = f32_to_f64(C.h[q + 1]) + f32_to_f64(C.l[q + 1]);
      }
    }
    split_x(px, U);
    split_f(pf, fh, fl);
  }

  __device__ __forceinline__ void store(const float (&v)[MC], int j) const {
    if constexpr (TRANS) {
      if (n < ldr) {
        TR* o = r + ((size_t)j * ldr + n) * M + m0;
        if constexpr (sizeof(TR) == 2) {
          const __nv_bfloat162 b0 = __floats2bfloat162_rn(v[0], v[1]), b1 = __floats2bfloat162_rn(v[2], v[3]);
          *reinterpret_cast<uint2*>(o) = make_uint2(bf2_u32(b0), bf2_u32(b1));
          if (sp == 2) {
            const float2 f0 = __bfloat1622float2(b0), f1 = __bfloat1622float2(b1);
            const __nv_bfloat162 c0 = __floats2bfloat162_rn(v[0] - f0.x, v[1] - f0.y);
            const __nv_bfloat162 c1 = __floats2bfloat162_rn(v[2] - f1.x, v[3] - f1.y);
            *reinterpret_cast<uint2*>(o + plane) = make_uint2(bf2_u32(c0), bf2_u32(c1));
          }
        } else {
          float hi[MC], lo[MC];
#pragma unroll
          for (int q = 0; q < MC; ++q) {
            hi[q] = sp == 2 ? __uint_as_float(__float_as_uint(v[q]) & 0xFFFFE000u) : v[q];
            lo[q] = v[q] - hi[q];
          }
          *reinterpret_cast<float4*>(o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
          if (sp == 2) *reinterpret_cast<float4*>(o + plane) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
    } else if (colok) {
      TR* o = r + ((size_t)j * M + m0) * K + n;
#pragma unroll
      for (int q = 0; q < MC; ++q) {
        if constexpr (sizeof(TR) == 8)
          o[(size_t)q * K] = f32_to_f64(v[q]);
        else
          o[(size_t)q * K] = v[q];
      }
    }
  }
};

// Runs when pass_lo <= st->solves <= pass_hi (the refinement's pass count).
template <typename TR, bool TRANS, int SRC>
__global__ void __launch_bounds__(256, 2) k_resid_dw(const double* __restrict__ F, const double* __restrict__ X,
                                                    const float* __restrict__ D1, const float* __restrict__ D2,
                                                    double* __restrict__ Xout, const float2* __restrict__ Cdw,
                                                    TR* __restrict__ r, int64_t N, int M, int64_t K, int64_t ldr,
                                                    int sp, int pass_lo, int pass_hi, IrState* st) {
  using W = DwResid<TR, TRANS, SRC>;
  constexpr int MC = W::MC, JC = W::JC;
  static_assert(SRC == 0 || TRANS, "the FP32 panels are block-transposed");
  if (st->done || st->solves < pass_lo || st->solves > pass_hi) return;
  W w;
  w.F = F;
  w.X = X;
  w.D1 = D1;
  w.D2 = D2;
  w.Xout = Xout;
  w.Cdw = Cdw;
  w.r = r;
  w.N = (int)N;
  w.K = (int)K;
  w.ldr = (int)ldr;
  w.M = M;
  w.sp = sp;
  w.plane = (size_t)N * ldr * M;
  const int lane = threadIdx.x % 32;
  const int tn = (int)(((TRANS ? ldr : K) + 31) / 32), tm = M / MC;
  const int64_t tj = (N + JC - 1) / JC;
  const int64_t nitem = tj * tm * tn;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t it = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; it < nitem; it += warps) {
    w.n = (int)(it % tn) * 32 + lane;
    w.m0 = (int)((it / tn) % tm) * MC;
    const int j0 = (int)(it / ((int64_t)tn * tm)) * JC;
    w.j1 = (int)min((int64_t)j0 + JC, N);
    w.colok = w.n < K;
    w.okl = w.colok && w.m0 > 0;
    w.okr = w.colok && w.m0 + MC < M;
    Slot<MC> A, B, C;
    float fh[MC], fl[MC];
    {
      typename W::Raw t;
      double tf[MC];
      w.load_x(j0 - 1, t);
      w.split_x(t, A);
      w.load_x(j0, t);
      w.split_x(t, B);
      w.load_x(j0 + 1, t);
      w.split_x(t, C);
      w.load_f(j0, tf);
      w.split_f(tf, fh, fl);
    }
    // rows (j-1, j, j+1) in (A, B, C), (B, C, A), (C, A, B) in turn
    for (int j = j0; j < w.j1; j += 3) {
      w.step(A, B, C, fh, fl, j);
      if (j + 1 < w.j1) w.step(B, C, A, fh, fl, j + 1);
      if (j + 2 < w.j1) w.step(C, A, B, fh, fl, j + 2);
    }
  }
  // |v| >= 2^77 (or non-finite) anywhere: the FP64 kernel recomputes
  if (__any_sync(0xffffffffu, w.amax >= (1100u << 21) || w.fbig) && lane == 0) atomicExch(&st->range, 1);
  block_add(w.acc.total(), &st->rn2[st->cur]);
}

// X from the row-major FP32 panels of the unit-stencil refinement: X = d1
// (+ d when D2 != NULL), exact in FP64.  Runs when pass_lo <= st->solves <=
// pass_hi and, with need_range, only if st->range is set (the double-word
// residual then hands over to the FP64 one, which reads X); ignores the stop
// flag (it also writes the final iterate once the refinement has stopped).
// Grid-stride over the N M K entries; consecutive threads, consecutive n.
__global__ void __launch_bounds__(256) k_x_from_panels(const float* __restrict__ D1, const float* __restrict__ D2,
                                                       double* __restrict__ X, size_t n, int pass_lo, int pass_hi,
                                                       int need_range, const IrState* st) {
  if (st->solves < pass_lo || st->solves > pass_hi || (need_range && !st->range)) return;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    X[e] = D2 != nullptr ? f32_to_f64(__ldg(D1 + e)) + f32_to_f64(__ldg(D2 + e)) : f32_to_f64(__ldg(D1 + e));
}

// X += d (row-major FP32 panel) for the later refinement passes of the
// unit-stencil flow (runs when st->solves >= pass_lo and the refinement has
// not stopped).
__global__ void __launch_bounds__(256) k_x_add_panel(const float* __restrict__ D, double* __restrict__ X, size_t n,
                                                     int pass_lo, const IrState* st) {
  if (st->done || st->solves < pass_lo) return;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    X[e] += f32_to_f64(__ldg(D + e));
}

// The first residual (X = 0): F rounded into the block-transposed panel, one
// warp per (block row, 16 rows m, 32 columns n); lane n writes 32 contiguous
// bytes per BF16 plane (a full 32-byte sector) and accumulates ||F||^2.
// HBM-bound: 8 bytes read and 2 sp (BF16) or 4 sp (FP32) bytes written per entry.
template <typename TR>
__global__ void __launch_bounds__(256) k_round_rhs(const double* __restrict__ F, TR* __restrict__ r, int64_t N, int M,
                                                   int Mr, int64_t K, int64_t Kp, int sp, IrState* st) {
  // Mr: rows per block row of the panel (M padded to the tensor-core tile;
  // rows past M are written as zeros)
  if (st->done) return;
  const size_t plane = (size_t)N * Kp * Mr;
  const int lane = threadIdx.x % 32;
  const int tn = (int)((Kp + 31) / 32), tm = Mr / 16;
  const int64_t nitem = N * tm * tn;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  Ssq acc;
  for (int64_t it = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; it < nitem; it += warps) {
    const int n = (int)(it % tn) * 32 + lane;
    const int m0 = (int)((it / tn) % tm) * 16;
    const int64_t j = it / ((int64_t)tn * tm);
    if (n >= Kp) continue;
    const double* fj = F + ((size_t)j * M + m0) * K + n;
    float v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      v[q] = (n < K && m0 + q < M) ? f64_to_f32_rz(fj[(size_t)q * K]) : 0.f;
      acc.add(v[q]);
    }
    TR* o = r + ((size_t)j * Kp + n) * Mr + m0;
    if constexpr (sizeof(TR) == 2) {
      uint32_t h[8], l[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        const float2 bf = __bfloat1622float2(b);
        const __nv_bfloat162 c = __floats2bfloat162_rn(v[2 * q] - bf.x, v[2 * q + 1] - bf.y);
        h[q] = *reinterpret_cast<const uint32_t*>(&b);
        l[q] = *reinterpret_cast<const uint32_t*>(&c);
      }
      reinterpret_cast<uint4*>(o)[0] = make_uint4(h[0], h[1], h[2], h[3]);
      reinterpret_cast<uint4*>(o)[1] = make_uint4(h[4], h[5], h[6], h[7]);
      if (sp == 2) {
        reinterpret_cast<uint4*>(o + plane)[0] = make_uint4(l[0], l[1], l[2], l[3]);
        reinterpret_cast<uint4*>(o + plane)[1] = make_uint4(l[4], l[5], l[6], l[7]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          hi[e] = sp == 2 ? __uint_as_float(__float_as_uint(v[4 * q + e]) & 0xFFFFE000u) : v[4 * q + e];
          lo[e] = v[4 * q + e] - hi[e];
        }
        reinterpret_cast<float4*>(o)[q] = make_float4(hi[0], hi[1], hi[2], hi[3]);
        if (sp == 2) reinterpret_cast<float4*>(o + plane)[q] = make_float4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
  }
  block_add(acc.total(), &st->fn2);
  block_add(acc.total(), &st->rn2[0]);
}

// r_j = F_j + A_j X_{j-1} + B_j X_{j+1} - C_j X_j with dense blocks, FP64.
// One CTA per (block row, column tile); a thread owns row m and CW columns.
// Output row-major (TRANS = false, leading dimension ldr) or block-transposed
// (TRANS = true, leading dimension ldr = Kp; columns K..Kp-1 written as zero).
template <typename TR, int CW, bool TRANS>
__global__ void k_resid_dense(const double* __restrict__ F, const double* __restrict__ X,
                              const double* __restrict__ A, const double* __restrict__ B,
                              const double* __restrict__ C, TR* __restrict__ r, int64_t N, int M, int64_t K,
                              int64_t ldr, int pass, int sp, IrState* st, int Mr) {
  // TRANS: the panel has Mr >= M rows per block row (rows past M get zeros)
  if (st->done) return;
  extern __shared__ double sm[];
  const int CG = blockDim.x / M, kt = CW * CG;
  const int t = threadIdx.x, m = t / CG, c0 = (t % CG) * CW;
  const int64_t j = blockIdx.x, col0 = (int64_t)blockIdx.y * kt, col = col0 + c0;
  const size_t MM = (size_t)M * M, MK = (size_t)M * K;
  double* xm = sm;
  double* x0 = sm + M * kt;
  double* xp = sm + 2 * M * kt;
  for (int e = t; e < M * kt; e += blockDim.x) {
    const int rr = e / kt, cc = e % kt;
    const int64_t cl = col0 + cc;
    const bool ok = cl < K;
    x0[e] = ok ? X[j * MK + (size_t)rr * K + cl] : 0.0;
    xm[e] = (ok && j > 0) ? X[(j - 1) * MK + (size_t)rr * K + cl] : 0.0;
    xp[e] = (ok && j + 1 < N) ? X[(j + 1) * MK + (size_t)rr * K + cl] : 0.0;
  }
  __syncthreads();
  double acc[CW];
  double part = 0.0;
  if (m < M) {
#pragma unroll
    for (int c = 0; c < CW; ++c) acc[c] = (col + c < K) ? F[j * MK + (size_t)m * K + col + c] : 0.0;
    const double* Ar = A + j * MM + (size_t)m * M;
    const double* Br = B + j * MM + (size_t)m * M;
    const double* Cr = C + j * MM + (size_t)m * M;
    for (int k = 0; k < M; ++k) {
      const double a = __ldg(Ar + k), b = __ldg(Br + k), cc = __ldg(Cr + k);
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        acc[c] = fma(a, xm[k * kt + c0 + c], acc[c]);
        acc[c] = fma(b, xp[k * kt + c0 + c], acc[c]);
        acc[c] = fma(-cc, x0[k * kt + c0 + c], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      const bool in = col + c < K;
      if (in) part += acc[c] * acc[c];
      if (TRANS) {
        if (col + c < ldr)
          put_planes(r, ((size_t)j * ldr + col + c) * Mr + m, (size_t)N * ldr * Mr, sp,
                     in ? f64_to_f32_rz(acc[c]) : 0.f);
      } else if (in) {
        r[j * (size_t)M * ldr + (size_t)m * ldr + col + c] = to_lp<TR>(acc[c]);
      }
    }
  }
  if (TRANS && Mr > M) {  // the padding rows of the tile's columns
    for (int e = t; e < (Mr - M) * kt; e += blockDim.x) {
      const int64_t cl = col0 + e / (Mr - M);
      if (cl < ldr) put_planes(r, ((size_t)j * ldr + cl) * Mr + M + e % (Mr - M), (size_t)N * ldr * Mr, sp, 0.f);
    }
  }
  (void)pass;
  block_add(part, &st->rn2[st->cur]);
}

// After every residual: records it, decides convergence (or a stall, or a
// tensor-core timeout), advances the slot, and -- inside the CUDA graph --
// sets the condition of the refinement loop: another pass runs while not
// done and fewer than max_it refinement solves have run.
// Per-set convergence (refined batches: column sets of one packed panel).
// After a residual (pass >= 1), k_col_ssq adds every column's sum of squares
// of the residual panel r into colssq (r as the next solve reads it: sp planes
// of TR, block-transposed [N][ldr][M] when trans, else row-major [N][M][ldr]);
// k_set_check reduces the columns to their sets, clears colssq, and sets
// st->setok when every set s has ||r_s||^2 <= tol2c ||F_s||^2 (tol2c: tol^2
// shrunk by the panel's rounding and the FP32 partial sums).
template <typename TR>
__global__ void __launch_bounds__(256) k_col_ssq(const TR* __restrict__ r, int sp, int trans, int64_t N, int M,
                                                 int64_t K, int64_t ldr, double* __restrict__ colssq,
                                                 const IrState* st) {
  if (st->done || st->cur == 0) return;
  const size_t plane = (size_t)N * ldr * M;
  const int64_t rows_per = (N + gridDim.y - 1) / gridDim.y;
  const int64_t j0 = (int64_t)blockIdx.y * rows_per, j1 = min(N, j0 + rows_per);
  if (trans) {
    // a column's M values of a block row are contiguous: one warp per column,
    // lanes along m (coalesced), 16 columns of the CTA's 128 per warp
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    for (int i = 0; i < 16; ++i) {
      const int64_t n = (int64_t)blockIdx.x * 128 + w * 16 + i;
      if (n >= K) break;
      double tot = 0.0;
      // four block rows per step, up to M / 32 <= 4 values of each per lane
      // and plane, all loads issued before the sums
      for (int64_t jb = j0; jb < j1; jb += 64) {
        float acc = 0.f;  // FP32 partial sums of at most 64 x 4 squares per lane
        const int64_t je = min(j1, jb + 64);
        for (int64_t j = jb; j < je; j += 4) {
          float v[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              v[u][q] = 0.f;
              if (j + u < je && lane + 32 * q < M) {
                const TR* e = r + ((size_t)(j + u) * ldr + n) * M + lane + 32 * q;
                v[u][q] = lp_to_float(e[0]);
                if (sp == 2) v[u][q] += lp_to_float(e[plane]);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc = fmaf(v[u][q], v[u][q], acc);
        }
        tot += acc;
      }
      for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
      if (lane == 0) atomicAdd(colssq + n, tot);
    }
    return;
  }
  // row-major: threads along n (coalesced), the two halves of the CTA split m
  const int64_t n = (int64_t)blockIdx.x * 128 + threadIdx.x % 128;
  if (n >= K) return;
  const int half = threadIdx.x / 128;
  float acc = 0.f;
  double tot = 0.0;
  int cnt = 0;
  for (int64_t j = j0; j < j1; ++j) {
    for (int m = half; m < M; m += 2) {
      const size_t e = ((size_t)j * M + m) * ldr + n;
      float v = 0.f;
      for (int p = 0; p < sp; ++p) v += lp_to_float(r[e + p * plane]);
      acc = fmaf(v, v, acc);
      if (++cnt == 256) {  // FP32 partial sums of at most 256 squares
        tot += acc;
        acc = 0.f;
        cnt = 0;
      }
    }
  }
  tot += acc;
  atomicAdd(colssq + n, tot);
}

__global__ void __launch_bounds__(256) k_set_check(double* __restrict__ colssq, const int* __restrict__ colset,
                                                   int64_t K, int nsets, const double* __restrict__ setn2,
                                                   double tol2c, IrState* st) {
  if (st->done || st->cur == 0) return;
  extern __shared__ double ss[];
  for (int s = threadIdx.x; s < nsets; s += blockDim.x) ss[s] = 0.0;
  __syncthreads();
  for (int64_t c = threadIdx.x; c < K; c += blockDim.x) {
    atomicAdd(ss + colset[c], colssq[c]);
    colssq[c] = 0.0;
  }
  __syncthreads();
  bool ok = true;
  for (int s = threadIdx.x; s < nsets; s += blockDim.x) {
    // ||F_s||^2 after the set's power-of-two scaling (set_exponent of the batch)
    const double n2 = setn2[s];
    int e = 0;
    if (n2 > 0.0 && n2 < INFINITY) frexp(sqrt(n2), &e);
    ok = ok && ss[s] <= tol2c * ldexp(n2, -2 * e);
  }
  ok = __syncthreads_and(ok);
  if (threadIdx.x == 0) st->setok = ok ? 1 : 0;
}

__global__ void k_ir_check(IrState* st, double tol2, int max_it, cudaGraphConditionalHandle loop, int setmode) {
  const int pass = st->cur;
  if (st->range) {  // the FP64 residual replaced the double-word one
    st->rn2[pass] = st->rn2_fb;
    st->rn2_fb = 0.0;
    st->range = 0;
  }
  if (!st->done) {
    st->last = pass;
    if (pass > 0) {
      const double r2 = st->rn2[pass];
      if (st->kstatus != 0) {
        st->done = 3;  // a tensor-core kernel gave up: stop, report
      } else if (setmode ? st->setok != 0 : r2 <= tol2 * st->fn2) {
        st->done = 1;
      } else if (pass >= 3 && r2 >= 0.9 * st->rn2[pass - 1] && st->rn2[pass - 1] >= 0.9 * st->rn2[pass - 2]) {
        st->done = 2;  // two passes without a 10 % reduction: stalled
      }
    }
  }
  st->cur = pass + 1;
  if (loop) cudaGraphSetConditional(loop, (st->done == 0 && pass >= 1 && pass < max_it + 1) ? 1u : 0u);
}

__global__ void k_count_solve(IrState* st) {
  if (!st->done) st->solves += 1;
}

template <typename Tin>
__global__ void k_cast(const double* __restrict__ src, Tin* __restrict__ dst, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (Tin)src[e];
}

bt_status grow(void** p, size_t* have, size_t need, cudaStream_t st) {
  if (need <= *have) return BT_OK;
  if (*p) {
    BT_CUDA(cudaStreamSynchronize(st));
    BT_CUDA(cudaFree(*p));
    *p = nullptr;
    *have = 0;
  }
  cudaError_t e = cudaMalloc(p, need);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error(std::string("refinement buffer allocation failed: ") + cudaGetErrorString(e));
    return BT_ERR_OOM;
  }
  *have = need;
  return BT_OK;
}

template <typename TR, bool TRANS, int SRC>
bt_status launch_dw(bt_handle_s* h, const double* F, const double* X, const float* d1, const float* d2, double* xout,
                    TR* r, int64_t K, int64_t ldr, int sp, int pass_lo, int pass_hi, IrState* st, cudaStream_t s) {
  using W = DwResid<TR, TRANS, SRC>;
  const int M = (int)h->M;
  static const int grid = resident_grid(reinterpret_cast<const void*>(&k_resid_dw<TR, TRANS, SRC>), 256, 0);
  const int64_t items = ((h->N + W::JC - 1) / W::JC) * (M / W::MC) * (((TRANS ? ldr : K) + 31) / 32);
  const int blocks = (int)std::min<int64_t>((items + 7) / 8, grid);
  k_resid_dw<TR, TRANS, SRC><<<blocks, 256, 0, s>>>(F, X, d1, d2, xout, reinterpret_cast<const float2*>(h->Cdw), r,
                                                     h->N, M, K, ldr, sp, pass_lo, pass_hi, st);
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

// The FP64 residual from X, run only if the double-word residual met an
// out-of-range value (gated on st->range; its norm goes to st->rn2_fb).
template <typename TR>
bt_status launch_fallback(bt_handle_s* h, const double* F, const double* X, TR* r, int64_t K, int64_t Kp, bool trans,
                          int sp, int pass, IrState* st, cudaStream_t s) {
  const int M = (int)h->M;
  ProfScope ps(h, s, "resid_fb");
  if (trans) {
    static const int grid = resident_grid(reinterpret_cast<const void*>(&k_resid_warp<TR>), 256, 0);
    const int64_t nwarp_items = h->N * (M / 8) * ((Kp + 31) / 32);
    const int blocks = (int)std::min<int64_t>((nwarp_items + 7) / 8, grid);
    k_resid_warp<TR><<<blocks, 256, 0, s>>>(F, X, h->Cdiag, r, h->N, M, M, K, Kp, pass, sp, st, &st->range);
  } else {
    const size_t n = (size_t)h->N * M * K;
    static const int grid = resident_grid(reinterpret_cast<const void*>(&k_resid_stencil<TR>), 256, 0);
    const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)grid);
    k_resid_stencil<TR><<<blocks, 256, 0, s>>>(F, X, h->Cdiag, r, h->N, M, K, 0, pass, st, &st->range);
  }
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

// X from the FP32 panels (k_x_from_panels), gated as that kernel describes.
bt_status launch_x_from_panels(bt_handle_s* h, const float* d1, const float* d2, double* X, int64_t K, int pass_lo,
                               int pass_hi, int need_range, const IrState* st, cudaStream_t s) {
  static const int grid = resident_grid(reinterpret_cast<const void*>(&k_x_from_panels), 256, 0);
  const size_t n = (size_t)h->N * h->M * K;
  k_x_from_panels<<<(int)std::min<size_t>((n + 255) / 256, (size_t)grid), 256, 0, s>>>(d1, d2, X, n, pass_lo,
                                                                                      pass_hi, need_range, st);
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

// The residuals of the unit-stencil refinement on the tensor-core panels,
// where the iterate lives in FP32 panels until the first refinement pass:
//   stage 1 (after the first solve): r = F - P d1 (X not written);
//   stage 2 (after a refinement solve d): on the first pass one kernel forms
//     X = d1 + d and r = F - P X from the panels; on later passes X += d,
//     then r from X.
// Either stage ends with the gated FP64 fallback.
template <typename TR>
bt_status launch_residual_panels(bt_handle_s* h, const double* F, double* X, const float* d1, const float* d,
                                 TR* r, int64_t K, int64_t Kp, int sp, IrState* st, int stage, cudaStream_t s) {
  const int M = (int)h->M;
  if (stage == 1) {
    {
      ProfScope ps(h, s, "resid_dw");
      BT_TRY((launch_dw<TR, true, 1>(h, F, nullptr, d1, nullptr, nullptr, r, K, Kp, sp, 0, 0, st, s)));
    }
    {
      ProfScope ps(h, s, "resid_fb");
      BT_TRY(launch_x_from_panels(h, d1, nullptr, X, K, 0, 0, 1, st, s));
    }
  } else {
    {
      ProfScope ps(h, s, "x_update");
      static const int grid = resident_grid(reinterpret_cast<const void*>(&k_x_add_panel), 256, 0);
      const size_t n = (size_t)h->N * M * K;
      k_x_add_panel<<<(int)std::min<size_t>((n + 255) / 256, (size_t)grid), 256, 0, s>>>(d, X, n, 2, st);
      BT_CUDA(cudaGetLastError());
    }
    ProfScope ps(h, s, "resid_dw");
    BT_TRY((launch_dw<TR, true, 0>(h, F, X, nullptr, nullptr, nullptr, r, K, Kp, sp, 2, INT32_MAX, st, s)));
    BT_TRY((launch_dw<TR, true, 2>(h, F, nullptr, d1, d, X, r, K, Kp, sp, 1, 1, st, s)));
  }
  return launch_fallback<TR>(h, F, X, r, K, Kp, true, sp, 0, st, s);
}

// Residual into the solve's panel: row-major (ld = K) for the SIMT solve,
// block-transposed (ld = Kp) for the tensor-core solve.
// rmode: 1 FP64 on the CUDA cores, 2 the tensor-core digit residual (dense
// blocks), 3 FP32 double-word arithmetic (unit stencils).
template <typename TR>
bt_status launch_residual(bt_handle_s* h, const double* F, const double* X, TR* r, int64_t K, int64_t Kp, bool trans,
                          int sp, int first, int pass, IrState* st, int rmode, cudaStream_t s) {
  const int M = (int)h->M;
  const int Mr = trans ? tc_M(h) : M;  // rows per block row of the tensor-core panel
  const bool digits = rmode == 2;
  if (digits && !first)  // dense blocks: the exact residual on the tensor cores
    return launch_resid_digits(h, F, X, K, trans ? 0 : 1, sizeof(TR) == 4, r, sp, &st->done, st->rn2, &st->cur,
                               &st->kstatus, s);
  // the first pass (X = 0) only rounds F into the panel: timed under its own name
  if (!first && rmode == 3) {
    // FP32 double-word residual; the FP64 kernel behind it runs only when a
    // value was out of its range (gated on st->range)
    {
      ProfScope ps(h, s, "resid_dw");
      if (trans)
        BT_TRY((launch_dw<TR, true, 0>(h, F, X, nullptr, nullptr, nullptr, r, K, Kp, sp, 0, INT32_MAX, st, s)));
      else
        BT_TRY((launch_dw<TR, false, 0>(h, F, X, nullptr, nullptr, nullptr, r, K, K, sp, 0, INT32_MAX, st, s)));
    }
    return launch_fallback<TR>(h, F, X, r, K, Kp, trans, sp, pass, st, s);
  }
  ProfScope ps(h, s, first ? "rhs_round" : "residual");
  if (first || h->stencil) {
    if (trans) {  // the tensor-core panels: Mr is 64 or 128
      if (first) {
        static const int grid = resident_grid(reinterpret_cast<const void*>(&k_round_rhs<TR>), 256, 0);
        const int64_t items = h->N * (Mr / 16) * ((Kp + 31) / 32);
        const int blocks = (int)std::min<int64_t>((items + 7) / 8, grid);
        k_round_rhs<TR><<<blocks, 256, 0, s>>>(F, r, h->N, M, Mr, K, Kp, sp, st);
      } else {
        static const int grid = resident_grid(reinterpret_cast<const void*>(&k_resid_warp<TR>), 256, 0);
        const int64_t nwarp_items = h->N * (Mr / 8) * ((Kp + 31) / 32);
        const int blocks = (int)std::min<int64_t>((nwarp_items + 7) / 8, grid);
        k_resid_warp<TR><<<blocks, 256, 0, s>>>(F, X, h->Cdiag, r, h->N, M, Mr, K, Kp, pass, sp, st, nullptr);
      }
    } else {
      const size_t n = (size_t)h->N * M * K;
      static const int grid = resident_grid(reinterpret_cast<const void*>(&k_resid_stencil<TR>), 256, 0);
      const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)grid);
      k_resid_stencil<TR><<<blocks, 256, 0, s>>>(F, X, h->Cdiag, r, h->N, M, K, first, pass, st, nullptr);
    }
  } else {
    constexpr int CW = 4;
    const int CG = std::max(1, std::min(1024 / M, std::max(1, 128 / M)));
    const int kt = CW * CG;
    const int64_t ncols = trans ? Kp : K;
    const int64_t ntiles = (ncols + kt - 1) / kt;
    const size_t smem = 3 * (size_t)M * kt * sizeof(double);
    if (trans) {
      if (smem > 48 * 1024)
        BT_CUDA(cudaFuncSetAttribute(k_resid_dense<TR, CW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_resid_dense<TR, CW, true><<<dim3((unsigned)h->N, (unsigned)ntiles), M * CG, smem, s>>>(
          F, X, h->A, h->B, h->C, r, h->N, M, K, Kp, pass, sp, st, Mr);
    } else {
      if (smem > 48 * 1024)
        BT_CUDA(cudaFuncSetAttribute(k_resid_dense<TR, CW, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_resid_dense<TR, CW, false><<<dim3((unsigned)h->N, (unsigned)ntiles), M * CG, smem, s>>>(
          F, X, h->A, h->B, h->C, r, h->N, M, K, K, pass, 1, st, M);
    }
  }
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

}  // namespace

bool resid_dw_supported(const bt_handle_s* h) { return h->stencil && h->stencil_unit && h->M % 8 == 0; }

bt_status make_f32_factors(bt_handle_s* h, cudaStream_t st) {
  LowFactors& f = h->f32;
  if (f.ready) return BT_OK;
  const size_t MM = (size_t)h->M * h->M, NB = (size_t)h->N * MM, SB = (size_t)h->S * MM;
  DevArena& ar = h->arena;
  struct Item {
    float** dst;
    const double* src;
    size_t n;
  } items[] = {{&f.Dinv, h->Dinv, NB}, {&f.E, h->E, NB},   {&f.G, h->G, NB},   {&f.U, h->U, NB},
               {&f.V, h->V, NB},       {&f.AK, h->AK, SB}, {&f.BK, h->BK, SB}, {&f.R, h->R, (size_t)h->depth * SB},
               {&f.HL, h->HL, SB},     {&f.HR, h->HR, SB}};
  for (auto& it : items) {
    BT_TRY(ar.alloc((void**)it.dst, it.n * sizeof(float)));
    k_cast<float><<<1024, 256, 0, st>>>(it.src, *it.dst, it.n);
  }
  BT_CUDA(cudaGetLastError());
  f.ready = true;
  return BT_OK;
}

bt_status solve_refined(bt_handle_s* h, const double* F, int64_t K, double* X, const bt_opts& o, bt_info* info,
                        int how, cudaStream_t rec, const SetCheck* sc) {
  cudaStream_t s = (cudaStream_t)o.stream;
  const int gen0 = h->lp_gen;
  // default passes: the split-BF16 solve gains about five digits per pass, the
  // single-plane precisions about two to three
  const int max_it = o.max_it > 0 ? std::min(o.max_it, kMaxPasses - 3) : (o.precision == BT_PREC_BF16X3 ? 6 : 12);
  const double tol = o.tol > 0 ? o.tol : 1e-10;
  const int prec = o.precision;
  const bool tcore = prec == BT_PREC_BF16 || prec == BT_PREC_TF32 || prec == BT_PREC_BF16X3;
  const int sp = tcore ? tc_planes(prec) : 1;
  const int M = (int)h->M;
  // rows per block row of the low-precision panels: the tensor-core tile
  // (64 or 128, zero padding past M), else M
  const int Mt = tcore ? tc_M(h) : M;
  int64_t Kp = K;
  size_t eb = sizeof(float);
  if (tcore) {
    const int nt = tc_col_tile(prec, M);
    if (nt == 0 || Mt == 0) {
      set_error("bt_solve_ex: the tensor-core precisions support block sizes M <= 128");
      return BT_ERR_UNSUPPORTED;
    }
    Kp = (K + nt - 1) / nt * nt;
    eb = prec == BT_PREC_TF32 ? 4 : 2;
  }
  // residual: 0 automatic (the tensor-core digit residual for dense blocks,
  // the FP32 double-word residual for unit stencils, where they apply), 1 FP64
  // on the CUDA cores, 2 the tensor-core digit residual, 3 double-word
  const bool dig_ok = resid_digits_supported(h, K);
  // the double-word residual writes unpadded tensor-core panels
  const bool dw_ok = resid_dw_supported(h) && (!tcore || Mt == M);
  if (o.residual == 2 && !dig_ok) {
    set_error("bt_solve_ex: the tensor-core residual needs dense blocks with M = 64 or M = 128");
    return BT_ERR_UNSUPPORTED;
  }
  if (o.residual == 3 && !dw_ok) {
    set_error("bt_solve_ex: the double-word residual needs A_j = B_j = I, C_j = tridiag(-1, c, -1) with "
              "2^-30 <= |c| <= 2^30, and M a multiple of 8 (64 or 128 with the tensor-core precisions)");
    return BT_ERR_UNSUPPORTED;
  }
  const bool digits = o.residual == 2 || (o.residual == 0 && dig_ok);
  const int rmode = digits ? 2 : (o.residual == 3 || (o.residual == 0 && dw_ok)) ? 3 : 1;
  // unit stencils on the tensor-core panels: the first solve's result stays an
  // FP32 panel (d1) and the first refinement pass forms X = d1 + d together
  // with its residual (launch_residual_panels)
  const bool pairflow = tcore && rmode == 3 && prec == BT_PREC_BF16X3 && M == 128;
  const void* before[5] = {h->lp_r, h->lp_d, h->lp_c, h->lp_x, h->lp_x1};
  const size_t panel = (size_t)sp * h->N * Mt * Kp * eb;
  // series terms [depth][S] and, for the tensor-core step 2.2, one node sum per tree node
  const size_t cbytes = ((size_t)h->depth * h->S + h->nodes.size()) * Mt * Kp * sizeof(float);
  BT_TRY(grow(&h->lp_r, &h->lp_panel_bytes, panel, s));
  BT_TRY(grow(&h->lp_d, &h->lp_d_bytes, panel, s));
  BT_TRY(grow(&h->lp_c, &h->lp_c_bytes, cbytes, s));
  if (tcore) BT_TRY(grow(&h->lp_x, &h->lp_x_bytes, (size_t)h->N * Mt * Kp * sizeof(float), s));
  if (pairflow) BT_TRY(grow(&h->lp_x1, &h->lp_x1_bytes, (size_t)h->N * M * K * sizeof(float), s));
  if (before[0] != h->lp_r || before[1] != h->lp_d || before[2] != h->lp_c || before[3] != h->lp_x ||
      before[4] != h->lp_x1)
    ++h->lp_gen;
  if (!h->ir_state) BT_CUDA(cudaMalloc(&h->ir_state, sizeof(IrState)));
  if (digits) BT_TRY(resid_digits_prepare(h, K, s));
  BT_TRY(make_f32_factors(h, s));
  if (tcore) BT_TRY(make_tc_factors(h, prec, s));
  if (!h->rg_cap2) BT_CUDA(cudaStreamCreateWithFlags(&h->rg_cap2, cudaStreamNonBlocking));
  if (how == 2 && h->lp_gen != gen0) {
    set_error("refinement recorded into a capture before its buffers were prepared");
    return BT_ERR_ARG;
  }
  IrState* st = reinterpret_cast<IrState*>(h->ir_state);
  const int* done = &st->done;
  const double tol2 = tol * tol;

  // The refinement as a prologue (F rounded, first solve, first residual and
  // check) and a body (one refinement pass: solve, update, residual, check).
  // Launched directly, the body is unrolled max_it times and passes after
  // convergence return at once; in the CUDA graph it is the body of a
  // device-side WHILE node whose condition the check kernel sets.
  float* d1 = reinterpret_cast<float*>(h->lp_x1);
  float* dk = reinterpret_cast<float*>(h->lp_x);
  // first: 1 the first residual (X = 0: F rounded), else 0; stage: 1 after the
  // first solve, 2 after a refinement solve
  auto residual = [&](cudaStream_t q, int first, int stage) -> bt_status {
    if (pairflow && !first) {
      if (prec == BT_PREC_TF32)
        return launch_residual_panels<float>(h, F, X, d1, dk, reinterpret_cast<float*>(h->lp_r), K, Kp, sp, st,
                                             stage, q);
      return launch_residual_panels<__nv_bfloat16>(h, F, X, d1, dk, reinterpret_cast<__nv_bfloat16*>(h->lp_r), K,
                                                   Kp, sp, st, stage, q);
    }
    if (prec == BT_PREC_BF16 || prec == BT_PREC_BF16X3)
      return launch_residual<__nv_bfloat16>(h, F, X, reinterpret_cast<__nv_bfloat16*>(h->lp_r), K, Kp, true, sp,
                                            first, 0, st, rmode, q);
    return launch_residual<float>(h, F, X, reinterpret_cast<float*>(h->lp_r), K, Kp, tcore, sp, first, 0, st, rmode,
                                  q);
  };
  auto inner = [&](cudaStream_t q, int accumulate) -> bt_status {
    if (tcore) {
      TcBuffers tb{prec == BT_PREC_BF16 ? h->tc_fac_bf16 : prec == BT_PREC_TF32 ? h->tc_fac_tf32 : h->tc_fac_bf16x3,
                   h->lp_r, h->lp_d, reinterpret_cast<float*>(h->lp_c), dk, Kp,
                   pairflow ? (accumulate == 0 ? d1 : dk) : nullptr};
      // the panel flow keeps the solves' results in the FP32 panels (mode 2)
      return solve_tc(h, prec, tb, K, X, pairflow ? 2 : accumulate, done, &st->kstatus, q);
    }
    return solve_simt_f32(h, reinterpret_cast<float*>(h->lp_r), K, reinterpret_cast<float*>(h->lp_d),
                          reinterpret_cast<float*>(h->lp_c), X, accumulate, done, q);
  };
  auto check = [&](cudaStream_t q, cudaGraphConditionalHandle loop) {
    ProfScope ps(h, q, "ir_check");
    if (sc != nullptr) {
      // the panel's relative rounding u (BF16 2^-8, TF32 2^-11, split BF16
      // about 2^-16, FP32 rounded toward zero 2^-23), with a factor 2 to spare
      const double u = prec == BT_PREC_BF16 ? 0x1p-7 : prec == BT_PREC_TF32 ? 0x1p-10
                       : prec == BT_PREC_BF16X3 ? 0x1p-15 : 0x1p-22;
      const double tol2c = tol2 * (1.0 - u) * (1.0 - u) * (1.0 - 0x1p-12);
      const int64_t ldr = tcore ? Kp : K;
      const int64_t tiles = (K + 127) / 128;
      const dim3 g((unsigned)tiles, (unsigned)std::max<int64_t>(1, std::min<int64_t>(h->N, 2432 / tiles)));
      if (prec == BT_PREC_BF16 || prec == BT_PREC_BF16X3)
        k_col_ssq<__nv_bfloat16><<<g, 256, 0, q>>>(reinterpret_cast<const __nv_bfloat16*>(h->lp_r), sp, tcore ? 1 : 0,
                                                   h->N, Mt, K, ldr, sc->colssq, st);
      else
        k_col_ssq<float><<<g, 256, 0, q>>>(reinterpret_cast<const float*>(h->lp_r), sp, tcore ? 1 : 0, h->N, Mt, K,
                                           ldr, sc->colssq, st);
      k_set_check<<<1, 256, (size_t)sc->nsets * sizeof(double), q>>>(sc->colssq, sc->colset, K, sc->nsets, sc->n2,
                                                                    tol2c, st);
    }
    k_ir_check<<<1, 1, 0, q>>>(st, tol2, max_it, loop, sc != nullptr ? 1 : 0);
  };
  auto prologue = [&](cudaStream_t q, cudaGraphConditionalHandle loop) -> bt_status {
    BT_CUDA(cudaMemsetAsync(st, 0, sizeof(IrState), q));
    BT_TRY(residual(q, 1, 0));
    check(q, 0);
    BT_TRY(inner(q, 0));
    BT_TRY(residual(q, 0, 1));
    check(q, loop);
    return BT_OK;
  };
  // after the refinement: with no refinement pass taken, the panel flow's
  // solution is still the FP32 panel d1
  auto epilogue = [&](cudaStream_t q) -> bt_status {
    if (!pairflow) return BT_OK;
    ProfScope ps(h, q, "x_update");
    return launch_x_from_panels(h, d1, nullptr, X, K, 0, 0, 0, st, q);
  };
  auto body = [&](cudaStream_t q, cudaGraphConditionalHandle loop) -> bt_status {
    {
      ProfScope ps(h, q, "ir_check");
      k_count_solve<<<1, 1, 0, q>>>(st);
    }
    BT_TRY(inner(q, 1));
    BT_TRY(residual(q, 0, 2));
    check(q, loop);
    return BT_OK;
  };
  auto enqueue = [&](cudaStream_t q) -> bt_status {
    BT_TRY(prologue(q, 0));
    for (int it = 0; it < max_it; ++it) BT_TRY(body(q, 0));
    BT_TRY(epilogue(q));
    BT_CUDA(cudaGetLastError());
    return BT_OK;
  };
  // Records prologue + WHILE(body) + epilogue into the capture in progress on
  // q (the WHILE body is captured on a second stream into the node's graph).
  auto record = [&](cudaStream_t q) -> bool {
    cudaStream_t cap2 = h->rg_cap2;
    bool ok = true;
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    cudaGraphConditionalHandle loop = 0;
    ok = ok && cudaStreamGetCaptureInfo(q, &cs, nullptr, &cg) == cudaSuccess && cg != nullptr;
    ok = ok && cudaGraphConditionalHandleCreate(&loop, cg, 0, cudaGraphCondAssignDefault) == cudaSuccess;
    ok = ok && prologue(q, loop) == BT_OK;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    ok = ok && cudaStreamGetCaptureInfo(q, &cs, nullptr, &cg, &deps, nullptr, &nd) == cudaSuccess;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn = nullptr;
    ok = ok && cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &cp) == cudaSuccess;
    ok = ok && cudaStreamUpdateCaptureDependencies(q, &cn, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                   cudaSuccess;
    if (ok) {
      cudaGraph_t bg = cp.conditional.phGraph_out[0];
      ok = cudaStreamBeginCaptureToGraph(cap2, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
           cudaSuccess;
      if (ok) {
        const bt_status bs = body(cap2, loop);
        cudaGraph_t bg_out = nullptr;
        ok = cudaStreamEndCapture(cap2, &bg_out) == cudaSuccess && bs == BT_OK;
      }
    }
    return ok && epilogue(q) == BT_OK;  // after the WHILE node
  };
  if (how == 1) {  // one direct run builds what the launches build lazily (job tables, scratch)
    BT_TRY(enqueue(s));
    BT_CUDA(cudaStreamSynchronize(s));
    return BT_OK;
  }
  if (how == 2) {
    if (!record(rec)) {
      set_error("refinement: recording into the capture failed");
      return BT_ERR_CUDA;
    }
    return BT_OK;
  }
  // Captures the refinement into *out; false (and nothing captured) on failure.
  auto capture = [&](cudaGraph_t* out) -> bool {
    cudaStream_t& cap = h->rg_cap;
    if (!cap && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    const bool ok = record(cap);
    cudaGraph_t graph = nullptr;
    const bool ended = cudaStreamEndCapture(cap, &graph) == cudaSuccess;
    if (!(ok && ended && graph)) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return false;
    }
    *out = graph;
    return true;
  };

  // CUDA graphs: a key's second call captures (the first has grown every
  // buffer and built every factor copy), later calls replay.  Profiling
  // records events per launch, so it runs the launches directly.
  auto& cache = h->rgraphs;
  auto drop = [](bt_handle_s::RefineGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g.exec = nullptr;
    g.graph = nullptr;
  };
  for (size_t i = 0; i < cache.size();) {  // graphs of buffers that have moved
    if (cache[i].gen != h->lp_gen) {
      drop(cache[i]);
      cache.erase(cache.begin() + (std::ptrdiff_t)i);
    } else {
      ++i;
    }
  }
  const int rkey = rmode;
  bt_handle_s::RefineGraph* e = nullptr;
  for (auto& g : cache)
    if (g.F == F && g.X == X && g.K == K && g.precision == prec && g.tol == tol && g.max_it == max_it &&
        g.resid == rkey) {
      e = &g;
      break;
    }
  bool launched = false;
  if (e != nullptr && !h->prof.on && !h->rg_broken) {
    if (!e->exec) {
      cudaGraph_t graph = nullptr;
      bool ok = capture(&graph);
      ok = ok && cudaGraphInstantiate(&e->exec, graph, 0) == cudaSuccess;
      if (ok) {
        e->graph = graph;
      } else {
        if (graph) cudaGraphDestroy(graph);
        e->exec = nullptr;
        h->rg_broken = true;
        cudaGetLastError();
      }
    }
    if (e->exec) {
      BT_CUDA(cudaGraphLaunch(e->exec, s));
      launched = true;
    }
  }
  if (!launched) BT_TRY(enqueue(s));
  if (e == nullptr) {
    if (cache.size() >= bt_handle_s::kMaxRefineGraphs) {
      auto lru = std::min_element(cache.begin(), cache.end(),
                                  [](const bt_handle_s::RefineGraph& a, const bt_handle_s::RefineGraph& b) {
                                    return a.used < b.used;
                                  });
      drop(*lru);
      cache.erase(lru);
    }
    bt_handle_s::RefineGraph g;
    g.F = F;
    g.X = X;
    g.K = K;
    g.precision = prec;
    g.tol = tol;
    g.max_it = max_it;
    g.gen = h->lp_gen;
    g.resid = rkey;
    cache.push_back(g);
    e = &cache.back();
  }
  e->used = ++h->rg_clock;
  BT_CUDA(cudaGetLastError());
  if (info) {
    IrState hs;
    BT_CUDA(cudaMemcpyAsync(&hs, st, sizeof(IrState), cudaMemcpyDeviceToHost, s));
    BT_CUDA(cudaStreamSynchronize(s));
    info->iters = hs.solves;
    info->converged = hs.done == 1 ? 1 : 0;
    info->rel_res = hs.fn2 > 0 ? std::sqrt(hs.rn2[hs.last] / hs.fn2) : 0.0;
    info->rel_res0 = hs.fn2 > 0 ? std::sqrt(hs.rn2[1] / hs.fn2) : 0.0;
    if (hs.kstatus != 0) {
      set_error("bt_solve_ex: a tensor-core kernel gave up a bounded wait (code " + std::to_string(hs.kstatus) + ")");
      return BT_ERR_TIMEOUT;
    }
    if (!info->converged) {
      set_error("bt_solve_ex: refinement stopped at relative residual " + std::to_string(info->rel_res));
      return BT_ERR_NOCONV;
    }
  }
  return BT_OK;
}

bt_status residual_diag(bt_handle_s* h, const double* F, const double* X, int64_t K, double* R, int method,
                        double* norm2, cudaStream_t s) {
  const bool dig_ok = resid_digits_supported(h, K);
  if (method == 0) method = dig_ok ? 2 : 1;
  if (method == 2 && !dig_ok) {
    set_error("bt_residual: the tensor-core residual needs dense blocks with M = 64 or M = 128");
    return BT_ERR_UNSUPPORTED;
  }
  const int M = (int)h->M;
  if (method == 3 && !resid_dw_supported(h)) {
    set_error("bt_residual: the double-word residual needs A_j = B_j = I, C_j = tridiag(-1, c, -1) with "
              "2^-30 <= |c| <= 2^30, and M a multiple of 8");
    return BT_ERR_UNSUPPORTED;
  }
  if (!h->ir_state) BT_CUDA(cudaMalloc(&h->ir_state, sizeof(IrState)));
  IrState* st = reinterpret_cast<IrState*>(h->ir_state);
  BT_CUDA(cudaMemsetAsync(st, 0, sizeof(IrState), s));
  if (method == 2) {
    BT_TRY(resid_digits_prepare(h, K, s));
    BT_TRY(launch_resid_digits(h, F, X, K, 2, false, R, 1, &st->done, st->rn2, nullptr, &st->kstatus, s));
  } else if (method == 3) {
    BT_TRY((launch_dw<double, false, 0>(h, F, X, nullptr, nullptr, nullptr, R, K, K, 1, 0, INT32_MAX, st, s)));
    const size_t n = (size_t)h->N * M * K;
    k_resid_stencil<double><<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(
        F, X, h->Cdiag, R, h->N, M, K, 0, 0, st, &st->range);
    BT_CUDA(cudaGetLastError());
  } else {
    if (h->stencil) {
      const size_t n = (size_t)h->N * M * K;
      k_resid_stencil<double><<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(
          F, X, h->Cdiag, R, h->N, M, K, 0, 0, st, nullptr);
    } else {
      constexpr int CW = 4;
      const int CG = std::max(1, std::min(1024 / M, std::max(1, 128 / M)));
      const int kt = CW * CG;
      const size_t smem = 3 * (size_t)M * kt * sizeof(double);
      if (smem > 48 * 1024)
        BT_CUDA(cudaFuncSetAttribute(k_resid_dense<double, CW, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
      k_resid_dense<double, CW, false><<<dim3((unsigned)h->N, (unsigned)((K + kt - 1) / kt)), M * CG, smem, s>>>(
          F, X, h->A, h->B, h->C, R, h->N, M, K, K, 0, 1, st, M);
    }
    BT_CUDA(cudaGetLastError());
  }
  IrState hs;
  BT_CUDA(cudaMemcpyAsync(&hs, st, sizeof(IrState), cudaMemcpyDeviceToHost, s));
  BT_CUDA(cudaStreamSynchronize(s));
  if (hs.kstatus != 0) {
    set_error("bt_residual: a tensor-core kernel gave up a bounded wait (code " + std::to_string(hs.kstatus) + ")");
    return BT_ERR_TIMEOUT;
  }
  if (norm2) *norm2 = hs.range ? hs.rn2_fb : hs.rn2[0];
  return BT_OK;
}

size_t refine_state_bytes() { return sizeof(IrState); }

// Fills *info from a copy of a handle's refinement state; returns the
// tensor-core status word (non-zero: a bounded wait gave up).
int refine_state_info(const void* state, bt_info* info) {
  const IrState& hs = *reinterpret_cast<const IrState*>(state);
  info->iters = hs.solves;
  info->converged = hs.done == 1 ? 1 : 0;
  info->rel_res = hs.fn2 > 0 ? std::sqrt(hs.rn2[hs.last] / hs.fn2) : 0.0;
  info->rel_res0 = hs.fn2 > 0 ? std::sqrt(hs.rn2[1] / hs.fn2) : 0.0;
  return hs.kstatus;
}

}  // namespace bt
