// Batched FP64-accurate block products on the tcgen05 tensor cores from BF16
// digit slices: the dense GEMMs of the factorisation (Algorithm 2, stage 1:
// the block sweep of eqs. sub1-sub3, the reduced system of eq. red1 and the
// rows of the tree inverses), M = 128.  GB300 issues FP64 at 2 FMA per clock
// per SM, so these products bound the factorisation; BF16 MMAs run about
// 1800x faster.
//
//   D_e = alpha X_e Y_e + beta Z_e      (every batch entry e; M x M row-major
//                                        FP64 blocks; alpha = +-1, beta 0 or 1)
//
// Balancing.  X Y = (X 2^T)(2^-T Y) for T = diag(t_k); with cx(k) and ry(k)
// the exponents (floor log2) of the largest |X[r][k]| over r and |Y[k][c]|
// over c, t_k = floor((ry(k) - cx(k)) / 2) evens out the two sides of every
// contraction index.  Scaling the contraction index by powers of two (X D,
// D^-1 Y: the unknowns of a block row scaled by D) changes t_k by exactly the
// opposite amount, so the digits below, and the product, do not change; an
// index whose column of X or row of Y is zero contributes nothing and is
// dropped.  Below, x and y are the balanced values x 2^t_k and 2^-t_k y.
//
// Digit split.  x = X[r][k] with max_k |X[r][k]| < 2^ex(r) is taken in fixed
// point f = round(x 2^(56 - ex)), |f| <= 2^56, written in balanced base 128,
//   f = sum_{p=0..7} a_p 128^(7-p),   |a_0| <= 128,  |a_p| <= 64 (p >= 1):
// integers of at most 8 significant bits, exact in BF16.  Y's columns take
// their own scales ey(c) and digits b_q the same way.  The split works on the
// significand bits alone (integer pipe), the balancing included.
//
// Products.  sum_k x y = 2^(ex + ey - 112) sum_{p,q} 128^(14 - p - q) sum_k a_p b_q
// (plus the operands' rounding).  The 36 pairs with p + q = d <= 7 accumulate
// into TMEM accumulator d; pairs with p + q >= 8 are dropped.  Accumulator d
// sums at most M (2 * 128 * 64 + 6 * 64 * 64) = 2.5 * 2^14 M = 5.2e6 < 2^24
// integers in magnitude (M = 128), so its FP32 accumulation is exact.  The
// MMAs take Y's digit tile as the A operand (128 output columns c as TMEM
// lanes, contraction k) and up to four of X's digit slices stacked as the B
// operand (64 output rows r each), so the slices p0.. of digit q land in TMEM
// columns 64 (q + p0) ...: one accumulator of 64 columns per level d.
//
// Combination.  hi = sum_{d<=3} c_d 128^(3-d), lo = sum_{d>=4} c_d 128^(7-d)
// (both below 2^44: exact in int64 and in FP64), T = fl(hi 2^28 + lo) =
// fl(sum_d c_d 128^(7-d)), and since level d weighs 128^(14-d) 2^(ex+ey-112),
// D = alpha T 2^(ex + ey - 63) + beta Z.  Error per entry against the exact
// product sum_k X[r][k] Y[k][c]: the operands' fixed-point rounding (at most
// 2^(ex + ey - 56) per term), the dropped pairs (at most 2^12 sum_{d=8..14}
// (15 - d) 128^(14 - d) < 7.05 2^54 units of 2^(ex + ey - 112), i.e.
// 1.77 2^(ex + ey - 56) per term) and the rounding of T (at most
// 2^-53 M 2^(ex + ey)): in all below M 2^(ex(r) + ey(c) - 52), an FP64-level
// bound relative to M max_k |X[r][k] 2^t_k| max_k |2^-t_k Y[k][c]|
// (>= M 2^(ex + ey - 2)),
// before the final alpha / beta step's one rounding.  The bound and the
// exactness of every accumulator are pinned on the CPU with exact integer
// arithmetic (tests/test_digit_gemm_model.py).  A row or column holding a
// NaN or an infinity gives NaN entries.
//
//   k_gdig_prep   per entry (a cluster of four CTAs, a quarter each): t from
//                 the column maxima of X and the row maxima of Y, X digits
//                 [E][8][M][M] (row r, contraction k) with ex, Y digits
//                 [E][8][M][M] (column c, contraction k) with ey
//   k_gemm_digits one CTA per (entry, 64-row half): TMA warp = MMA thread,
//                 TMEM allocator warp, 8 epilogue warps

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <string>

#include "bt_internal.cuh"
#include "tc_ptx.cuh"

namespace bt {

namespace {

using namespace tc;

constexpr int GM = 128;                  // block size
constexpr int GD = 8;                    // digits per value
constexpr int GFB = 56;                  // fixed-point fraction bits
constexpr int XS = 64 * 128;             // one X digit slice in smem: 64 rows x 64 contraction values (bytes)
constexpr int YT = 128 * 128;            // one Y digit tile: 128 columns x 64 contraction values (bytes)
constexpr int GTHREADS = 64 + 256;       // issuing warp, TMEM warp, 8 epilogue warps
constexpr int GACC = 64;                 // TMEM columns per accumulator (64 output rows)
constexpr int GTMEM = GD * GACC;         // 512
constexpr uint32_t GCHUNK = GD * XS + GD * YT;  // bytes of one contraction chunk (both operands)
constexpr size_t GSMEM = 1024 + (size_t)GCHUNK + 8 * 3 + 16;
constexpr int kBadExp = 0x7FFF;          // scale of a row / column holding a NaN or an infinity

static_assert(GSMEM <= 227 * 1024, "shared memory per CTA");
static_assert(GTMEM <= 512, "accumulators fit in TMEM");

// round(v 2^(56 - e)) for |v| < 2^e, on the integer pipe: the significand
// shifted into place, rounded to nearest with ties to even (GB300 issues
// FP64 operations, conversions included, at 1/64 of its integer rate).
__device__ __forceinline__ long long fixed56(double v, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (be != 0) m |= 1ull << 52;
  // v = m 2^(max(be, 1) - 1075), so f = m 2^sh with sh <= 3 (|f| < 2^56)
  const int sh = (be != 0 ? be : 1) - 1075 + GFB - e;
  unsigned long long q;
  if (sh >= 0) {
    q = m << sh;
  } else if (-sh > 54) {
    q = 0;
  } else {
    const int t = -sh;
    q = m >> t;
    const unsigned long long rem = m & ((1ull << t) - 1), half = 1ull << (t - 1);
    q += (rem > half || (rem == half && (q & 1))) ? 1 : 0;
  }
  return (b >> 63) ? -(long long)q : (long long)q;
}

// A small integer (|r| < 2^22) as the bits of an FP32 value without a
// conversion instruction: r + 1.5 2^23 in the bits, minus 1.5 2^23 (exact).
__device__ __forceinline__ uint32_t small_int_f32_bits(int r) {
  return __float_as_uint(__int_as_float(0x4B400000 + r) - 12582912.0f);
}

// The 8 balanced base-128 digits of round(v 2^(56 - e)) (|v| < 2^e), each as
// FP32 bits; every digit (|d| <= 128) is exact in BF16, whose bits are the
// upper half of the FP32 ones.
__device__ __forceinline__ void digits8(double v, int e, uint32_t (&d)[GD]) {
  long long f = fixed56(v, e);
#pragma unroll
  for (int p = GD - 1; p >= 1; --p) {
    const int r = (int)((f + 64) & 127) - 64;
    d[p] = small_int_f32_bits(r);
    f = (f - r) >> 7;
  }
  d[0] = small_int_f32_bits((int)f);
}

// Four digits (FP32 bits, exact in BF16) packed as four BF16 values.
__device__ __forceinline__ uint2 pack_bf16x4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  return make_uint2(__byte_perm(a, b, 0x7632), __byte_perm(c, d, 0x7632));
}

constexpr int kNoExp = -0x40000000;     // exponent of a zero (or skipped) value: below every other
constexpr int kDropT = 0x40000000;      // t_k of a contraction index that contributes nothing

__device__ __forceinline__ bool bits_nonfinite(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7FF) == 0x7FF;
}

// floor(log2 |v|) from the bits (subnormals included); kNoExp for a zero, a
// NaN or an infinity.  No FP64 instruction.
__device__ __forceinline__ int exp_floor(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
  const int be = (int)(b >> 52);
  if (b == 0 || be == 0x7FF) return kNoExp;
  if (be != 0) return be - 1023;
  return -1023 - __clzll((long long)(b << 12));  // subnormal: the leading bit of the fraction
}

__device__ __forceinline__ int warp_max_int(int m) {
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}

// The scale e of a row of X (column of Y) with every balanced |value| < 2^e
// (that of frexp of the largest): 0 for an all-zero row, kBadExp if the row
// holds a NaN or an infinity.
__device__ __forceinline__ int scale_from_max(int m, bool bad) {
  if (bad) return kBadExp;
  return m == kNoExp ? 0 : m + 1;
}

// The digits of both operands of entry e on a cluster of four CTAs, a
// quarter q of each operand per CTA (512 threads).  (1) CTA q reads rows
// 32 q .. 32 q + 31 of X_e (kept in registers) and columns 32 q .. 32 q + 31 of
// Y_e (staged in shared memory) and forms the partial column maxima of X and
// row maxima of Y over them; (2) the four partials meet through distributed
// shared memory: t_k for every k; (3) the rows of X: a warp per row, its
// scale and 8 digit rows; (4) the columns of Y: a warp per column, its scale
// and 8 digit rows (contraction k contiguous).
constexpr int GPREP = 512;
__global__ void __launch_bounds__(GPREP) k_gdig_prep(const double* const* __restrict__ tab, __nv_bfloat16* __restrict__ Xd,
                                                     __nv_bfloat16* __restrict__ Yd, int* __restrict__ ex,
                                                     int* __restrict__ ey) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double ys[GM][33];
  __shared__ int cxw[GPREP / 32][GM];
  __shared__ int cxq[GM], ryq[GM];  // this CTA's partial maxima (read by the others)
  __shared__ int tks[GM];
  const int e = blockIdx.x / 4, q = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid % 32, w = tid / 32;
  constexpr int NW = GPREP / 32;
  static_assert(2 * NW == 32, "two rows of X per warp");
  const double* X = tab[4 * e];
  const double* Y = tab[4 * e + 1];
  // (1) rows 32 q + 2 w + h of X in registers (columns 4 lane .. 4 lane + 3)
  double v[2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = 32 * q + 2 * w + h;
#pragma unroll
    for (int i = 0; i < 4; ++i) v[h][i] = X[(size_t)r * GM + 4 * lane + i];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) cxw[w][4 * lane + i] = max(exp_floor(v[0][i]), exp_floor(v[1][i]));
  for (int i = tid; i < GM * 32; i += GPREP) ys[i / 32][i % 32] = Y[(size_t)(i / 32) * GM + 32 * q + i % 32];
  __syncthreads();
  if (tid < GM) {
    int a = kNoExp;
#pragma unroll
    for (int g = 0; g < NW; ++g) a = max(a, cxw[g][tid]);
    cxq[tid] = a;
    int b = kNoExp;
    for (int j = 0; j < 32; ++j) b = max(b, exp_floor(ys[tid][j]));
    ryq[tid] = b;
  }
  // (2) every CTA's partials published: t_k = floor((ry_k - cx_k) / 2)
  cl.sync();
  if (tid < GM) {
    int a = kNoExp, b = kNoExp;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      a = max(a, cl.map_shared_rank(cxq, r)[tid]);
      b = max(b, cl.map_shared_rank(ryq, r)[tid]);
    }
    tks[tid] = (a == kNoExp || b == kNoExp) ? kDropT : (b - a) >> 1;  // floor
  }
  __syncthreads();
  const int t[4] = {tks[4 * lane], tks[4 * lane + 1], tks[4 * lane + 2], tks[4 * lane + 3]};  // k = 4 lane + i
  // (3) rows of X: x 2^t
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = 32 * q + 2 * w + h;
    int m = kNoExp;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      bad = bad || bits_nonfinite(v[h][i]);
      const int x = exp_floor(v[h][i]);
      if (x != kNoExp && t[i] != kDropT) m = max(m, x + t[i]);
    }
    m = warp_max_int(m);
    bad = __any_sync(0xffffffffu, bad);
    const int es = scale_from_max(m, bad);
    if (lane == 0) ex[(size_t)e * GM + r] = es;
    uint32_t d[4][GD];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (bad || t[i] == kDropT) {
#pragma unroll
        for (int p = 0; p < GD; ++p) d[i][p] = 0u;
      } else {
        digits8(v[h][i], es - t[i], d[i]);  // round(v 2^t 2^(56 - es))
      }
    }
#pragma unroll
    for (int p = 0; p < GD; ++p)
      *reinterpret_cast<uint2*>(Xd + (((size_t)e * GD + p) * GM + r) * GM + 4 * lane) =
          pack_bf16x4(d[0][p], d[1][p], d[2][p], d[3][p]);
  }
  // (4) columns of Y: 2^-t y
  for (int j = w; j < 32; j += NW) {
    double y[4];  // rows 4 lane .. 4 lane + 3 of column 32 q + j
    int m = kNoExp;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      y[i] = ys[4 * lane + i][j];
      bad = bad || bits_nonfinite(y[i]);
      const int x = exp_floor(y[i]);
      if (x != kNoExp && t[i] != kDropT) m = max(m, x - t[i]);
    }
    m = warp_max_int(m);
    bad = __any_sync(0xffffffffu, bad);
    const int es = scale_from_max(m, bad);
    const int c = 32 * q + j;
    if (lane == 0) ey[(size_t)e * GM + c] = es;
    uint32_t d[4][GD];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (bad || t[i] == kDropT) {
#pragma unroll
        for (int p = 0; p < GD; ++p) d[i][p] = 0u;
      } else {
        digits8(y[i], es + t[i], d[i]);  // round(v 2^-t 2^(56 - es))
      }
    }
#pragma unroll
    for (int p = 0; p < GD; ++p)
      *reinterpret_cast<uint2*>(Yd + (((size_t)e * GD + p) * GM + c) * GM + 4 * lane) =
          pack_bf16x4(d[0][p], d[1][p], d[2][p], d[3][p]);
  }
  cl.sync();  // no CTA leaves while a partner may still read its partial maxima
}

__global__ void __launch_bounds__(GTHREADS, 1)
    k_gemm_digits(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_y,
                  const double* const* __restrict__ tab, const int* __restrict__ ex, const int* __restrict__ ey,
                  double alpha, double beta, int* status) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* sX = sm;              // 8 X digit slices (64 rows each)
  uint8_t* sY = sm + GD * XS;    // 8 Y digit tiles (128 columns each)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + GCHUNK);
  uint64_t* full = bars;         // a contraction chunk has landed (phase = chunk)
  uint64_t* mdone = bars + 1;    // the MMAs of chunk 0 have read the buffers
  uint64_t* accf = bars + 2;     // every MMA has completed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 3);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int e = blockIdx.x / 2, h = blockIdx.x % 2;

  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(mdone, 1);
    mbar_init(accf, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, GTMEM);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tm_x);
      prefetch_tmap(&tm_y);
      bool ok = true;
      uint32_t loaded = 0;
      const uint64_t xdesc = smem_desc(smem_u32(sX), 16, 1024);
      const uint64_t ydesc = smem_desc(smem_u32(sY), 16, 1024);
      for (int kb = 0; kb < GM / 64 && ok; ++kb) {
        if (kb > 0) ok = mbar_wait(mdone, 0);  // the buffers are free again
        if (!ok) break;
        mbar_arrive_expect_tx(full, GCHUNK);
        for (int p = 0; p < GD; ++p) tma_load_2d(sX + p * XS, &tm_x, kb * 64, (e * GD + p) * GM + h * 64, full);
        for (int q = 0; q < GD; ++q) tma_load_2d(sY + q * YT, &tm_y, kb * 64, (e * GD + q) * GM, full);
        ++loaded;
        ok = mbar_wait(full, kb & 1);
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int q = 0; q < GD; ++q) {
          const uint64_t yd = ydesc + (uint64_t)((q * YT) >> 4);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            // slices p = 0 .. 7 - q (p + q <= 7), at most four per instruction
#pragma unroll
            for (int p0 = 0; p0 < GD - q; p0 += 4) {
              const int np = GD - q - p0 < 4 ? GD - q - p0 : 4;
              mma_f16(tmem + GACC * (q + p0), yd + 2 * ks, xdesc + (uint64_t)((p0 * XS) >> 4) + 2 * ks,
                      instr_desc(1, 0, 128, 64 * np), (kb == 0 && q == 0 && ks == 0) ? 0u : 1u);
            }
          }
        }
        mma_commit(kb + 1 < GM / 64 ? mdone : accf);
      }
      if (!ok) {
        atomicExch(status, 2);
        if (loaded > 0) mbar_wait(full, (loaded - 1) & 1);  // no exit with copies in flight
      }
    }
  } else if (warp >= 2) {
    const int qd = warp & 3, g = (warp - 2) >> 2;  // TMEM lane quarter, row group
    const uint32_t lane_base = (uint32_t)(32 * qd) << 16;
    const int c = 32 * qd + lane;                   // output column
    bool ok = mbar_wait(accf, 0);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
      if (lane == 0) atomicExch(status, 2);
    } else {
      tc_fence_after();
      const double* const* te = tab + 4 * e;
      const double* Z = te[2];
      double* D = const_cast<double*>(te[3]);
      const int eyc = ey[(size_t)e * GM + c];
#pragma unroll 1
      for (int k8 = 0; k8 < 4; ++k8) {
        const int rl = g * 32 + k8 * 8;  // first of this chunk's 8 rows within the half
        uint32_t a[32], b[32];
        tmem_ld8x4(tmem + lane_base + 0 * GACC + rl, tmem + lane_base + 1 * GACC + rl, tmem + lane_base + 2 * GACC + rl,
                   tmem + lane_base + 3 * GACC + rl, a);
        tmem_ld8x4(tmem + lane_base + 4 * GACC + rl, tmem + lane_base + 5 * GACC + rl, tmem + lane_base + 6 * GACC + rl,
                   tmem + lane_base + 7 * GACC + rl, b);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int r = h * 64 + rl + i;
          long long cd[GD];  // exact integers below 2^24: through int32 (FP32 pipe)
#pragma unroll
          for (int d = 0; d < 4; ++d) {
            cd[d] = (int)__uint_as_float(a[8 * d + i]);
            cd[d + 4] = (int)__uint_as_float(b[8 * d + i]);
          }
          const long long hi = ((cd[0] * 128 + cd[1]) * 128 + cd[2]) * 128 + cd[3];
          const long long lo = ((cd[4] * 128 + cd[5]) * 128 + cd[6]) * 128 + cd[7];
          const int exr = ex[(size_t)e * GM + r];
          const size_t o = (size_t)r * GM + c;
          double v;
          if (exr == kBadExp || eyc == kBadExp) {
            v = __longlong_as_double(0x7ff8000000000000LL);
          } else {
            // hi, lo (|x| < 2^44) as doubles exactly: x + 1.5 2^52 in the bits, minus 1.5 2^52
            const double dh = __longlong_as_double(0x4338000000000000LL + hi) - 6755399441055744.0;
            const double dl = __longlong_as_double(0x4338000000000000LL + lo) - 6755399441055744.0;
            const double t = fma(dh, 268435456.0, dl);
            // alpha 2^(ex + ey - 63): added to the exponent field and the sign bit (exact)
            // while the result stays a normal number, else through ldexp
            const int sx = exr + eyc - 2 * GFB + 7 * (GD - 1);
            const long long tb = __double_as_longlong(t);
            const int te = (int)((tb >> 52) & 0x7FF);
            if (te != 0 && te + sx > 0 && te + sx < 0x7FF) {
              v = __longlong_as_double((tb + (long long)sx * (1LL << 52)) ^ (alpha < 0.0 ? (long long)(1ULL << 63) : 0LL));
            } else {
              v = t == 0.0 ? 0.0 : alpha * ldexp(t, sx);
            }
          }
          if (beta != 0.0) v = fma(beta, Z[o], v);
          D[o] = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, GTMEM);
}

PFN_cuTensorMapEncodeTiled_v12000 gd_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  }
  return fn;
}

// 2-D BF16 map over rows x 128 contraction values, boxes of 64 values x box_rows, 128-byte swizzle.
bt_status gd_map(CUtensorMap* m, const void* base, uint64_t rows, uint32_t box_rows) {
  auto enc = gd_encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return BT_ERR_CUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)GM, rows};
  cuuint64_t strides[1] = {(cuuint64_t)GM * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return BT_ERR_CUDA;
  }
  return BT_OK;
}

}  // namespace

bool digit_gemm_supported(int M) { return M == GM; }

size_t digit_gemm_bytes(int emax) {
  return (size_t)emax * (2 * (size_t)GD * GM * GM * sizeof(__nv_bfloat16) + 2 * (size_t)GM * sizeof(int));
}

bt_status digit_gemm_run(void* scratch, int emax, const double* const* dtab, int E, double alpha, double beta,
                         int* status, cudaStream_t st) {
  if (E < 1 || E > emax) {
    set_error("digit GEMM: batch larger than its scratch");
    return BT_ERR_ARG;
  }
  __nv_bfloat16* Xd = reinterpret_cast<__nv_bfloat16*>(scratch);
  __nv_bfloat16* Yd = Xd + (size_t)emax * GD * GM * GM;
  int* ex = reinterpret_cast<int*>(Yd + (size_t)emax * GD * GM * GM);
  int* ey = ex + (size_t)emax * GM;
  CUtensorMap tx, ty;
  BT_TRY(gd_map(&tx, Xd, (uint64_t)E * GD * GM, 64));
  BT_TRY(gd_map(&ty, Yd, (uint64_t)E * GD * GM, 128));
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(4 * E));
    cfg.blockDim = dim3(GPREP);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 4;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    BT_CUDA(cudaLaunchKernelEx(&cfg, k_gdig_prep, dtab, Xd, Yd, ex, ey));
  }
  static bool attr = false;
  if (!attr) {
    BT_CUDA(cudaFuncSetAttribute(k_gemm_digits, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GSMEM));
    attr = true;
  }
  k_gemm_digits<<<(unsigned)(2 * E), GTHREADS, GSMEM, st>>>(tx, ty, dtab, ex, ey, alpha, beta, status);
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

}  // namespace bt
