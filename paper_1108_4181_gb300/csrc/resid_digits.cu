// Exact residual of the block-tridiagonal operator on the tcgen05 tensor cores.
//
//   r_j = F_j + A_j X_{j-1} + B_j X_{j+1} - C_j X_j      (the operator of
//   Section 2, dense M x M blocks, M = 64 or 128)
//
// Not in the paper: it is the FP64 residual of the iterative refinement around
// the low-precision stage 2, formed without FP64 arithmetic (this GPU issues
// FP64 at about 1/64 of its FP32 rate).
//
// Digit split.  A value v with |v| < 2^e is taken in fixed point with 49
// fraction bits, f = round(v 2^(49-e)), and f is written in balanced base 128,
//   f = sum_{p=0..6} a_p 128^(6-p),   |a_0| <= 128,  |a_p| <= 64 (p >= 1),
// so v = 2^e sum_p a_p 2^(-7(p+1)) to within 2^(e-50).  Every digit is an
// integer with at most 8 significant bits: exact in BF16.  The factor rows
// share one scale per block row j and row m (over A_j, B_j, -C_j: e_A(j,m)),
// the columns of X one scale per column over all block rows (e_X(n)).
//
// Products.  The digit pair (p, q) contributes a_p x_q 2^(e_A+e_X-14-7(p+q));
// the 28 pairs with p + q = d <= 6 accumulate into TMEM accumulator d (the
// pairs with p + q >= 7 lie below the fixed-point resolution and are dropped).
// An accumulator sums at most 3M (2*128*64 + 5*64*64) = 3M * 36864 <= 1.42e7
// < 2^24 in magnitude (M <= 128), and every addend is an integer, so the FP32
// accumulation is exact.  The MMAs use swapped roles: a 128-column tile of X
// digits is the A operand (M = 128 lanes = columns n), and the stacked digit
// slices of a factor block are the B operand (N = 64 per slice, up to four
// slices per instruction), so the accumulator of digit q and slices p0.. lands
// in TMEM columns 64 (q + p0) ...
//
// Combination.  In units u = 2^(e_A + e_X - 56):
//   T = sum_d c_d 128^(6-d)     (c_d the accumulators; int64, modulo 2^64)
//   R = round(F / u) + T        (modulo 2^64)
// equals the true r / u whenever |r| < 2^63 u; an FP32 estimate of F/u + T
// decides that (|estimate| < 2^62 with both terms below 2^83).  The remaining
// entries -- r large against the product scale (X far from a solution), or F
// non-finite -- take an FP64 path.  Error against the exact residual, per
// entry: at most 3M * 2.5 * 2^(e_A + e_X - 49) (fixed-point rounding of both
// operands and the dropped pairs) plus one unit u (F truncated to the unit).
//
//   k_fac_digits    factor digits [3N][7][M][M] and e_A (once per handle)
//   k_colmax        largest |X| of every column (its exponent)
//   k_x_digits      X digits, block-transposed [7][N][Kp][M], and e_X
//   k_resid_digits  persistent: TMA warp, MMA warp, 8 epilogue warps

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <string>

#include "bt_internal.cuh"
#include "tc_ptx.cuh"

namespace bt {

namespace {

using namespace tc;

constexpr int ND = 7;           // digits per value
constexpr int FB = 49;          // fixed-point fraction bits (7 digits of 7 bits)
constexpr int NX = 4;           // X-digit tile ring slots
constexpr int XT = 128 * 128;   // one X-digit tile: 128 columns x 64 contraction values (BF16)
constexpr int FSL = 64 * 128;   // one factor digit slice: 64 rows x 64 contraction values
constexpr int FST = ND * FSL;   // the 7 slices of one factor block and contraction chunk
constexpr int EGW = 2;          // epilogue warps per TMEM lane quarter (rows of an output half split EGW ways)
constexpr int RPT = 64 / EGW;   // output rows per epilogue thread
constexpr int THREADS = 64 + 128 * EGW;  // TMA warp, MMA warp, 4 EGW epilogue warps
constexpr int ACC = 64;         // TMEM columns of one accumulator
constexpr int TMEM_COLS = 512;  // 7 accumulators (448 columns)
constexpr int NBARS = 4 + 2 * NX + 3;
constexpr size_t SMEM = 1024 + 2 * (size_t)FST + NX * (size_t)XT + 8 * NBARS + 16;
constexpr int kBadScale = 0x7FFF;  // scale of a set holding a NaN or an infinity

static_assert(ND * ACC <= TMEM_COLS, "accumulators fit in TMEM");
static_assert(SMEM <= 227 * 1024, "shared memory per CTA");

// v = (-1)^neg * mant * 2^ex, be = biased exponent field
struct Dec {
  uint64_t mant;
  int ex, neg, be;
};

__device__ __forceinline__ Dec decode(double v) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  Dec d;
  d.neg = (int)(b >> 63);
  d.be = (int)((b >> 52) & 0x7FF);
  d.mant = b & 0xFFFFFFFFFFFFFull;
  if (d.be) {
    d.mant |= 1ull << 52;
    d.ex = d.be - 1075;
  } else {
    d.ex = -1074;
  }
  return d;
}

// 64-bit shifts whose amounts saturate at 64 (result 0), as PTX defines them.
__device__ __forceinline__ uint64_t shl64(uint64_t v, uint32_t n) {
  uint64_t r;
  asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(n));
  return r;
}
__device__ __forceinline__ uint64_t shr64(uint64_t v, uint32_t n) {
  uint64_t r;
  asm("shr.u64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(n));
  return r;
}

// e with |v| < 2^e for every v of a set whose largest magnitude has the bit
// pattern mx (sign cleared); 0 for an all-zero set, kBadScale for NaN / Inf.
__device__ __forceinline__ int scale_of(uint64_t mx) {
  if (mx == 0) return 0;
  const int be = (int)(mx >> 52);
  if (be >= 0x7FF) return kBadScale;
  return be == 0 ? -1022 : be - 1022;
}

// Balanced base-128 digits of round(v 2^(49-e)), |v| < 2^e; d[0] the most
// significant (|d[0]| <= 128, |d[p]| <= 64 otherwise).  The fixed-point value
// f is split once into f = hi 2^21 + lo (0 <= lo < 2^21); the three low digits
// come from lo, the borrow or carry they leave (0 or 1) moves into hi, and the
// four high digits come from hi -- 32-bit arithmetic throughout.
__device__ __forceinline__ void digits(double v, int e, int (&d)[ND]) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7FF);
  const uint64_t mant = (b & 0xFFFFFFFFFFFFFull) | (be ? (1ull << 52) : 0ull);
  const int r = e - (max(be, 1) - 1075) - FB;  // right shift that makes f (>= 4 for normal v)
  const uint64_t f = r <= 0 ? shl64(mant, (uint32_t)(-r))
                            : shr64(mant + shl64(1ull, (uint32_t)(r - 1)), (uint32_t)r);  // rounded
  const int64_t fs = (b >> 63) ? -(int64_t)f : (int64_t)f;
  int lo = (int)((uint64_t)fs & 0x1FFFFFull);
  int hi = (int)(fs >> 21);  // |f| <= 2^49
#pragma unroll
  for (int p = ND - 1; p > ND - 4; --p) {
    const int t = ((lo + 64) & 127) - 64;
    d[p] = t;
    lo = (lo - t) >> 7;
  }
  hi += lo;
#pragma unroll
  for (int p = ND - 4; p > 0; --p) {
    const int t = ((hi + 64) & 127) - 64;
    d[p] = t;
    hi = (hi - t) >> 7;
  }
  d[0] = hi;
}

// An integer |a| < 2^22 as FP32, exactly, without a conversion instruction.
__device__ __forceinline__ float small_int_f32(int a) { return __int_as_float(0x4B400000 + a) - 12582912.f; }

__device__ __forceinline__ uint32_t bf2(int a, int b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(small_int_f32(a), small_int_f32(b));
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }  // e in [-126, 127]

// x * 2^e for any e (two exact power-of-two factors, each within FP32 range).
__device__ __forceinline__ float scale_f(float x, int e) {
  const int e1 = max(-126, min(127, e));
  const int e2 = max(-126, min(127, e - e1));
  return x * pow2f(e1) * pow2f(e2);
}

// --------------------------------------------------------------- preparation
// One warp per (block row j, row m): the scale of row m over A_j, B_j and C_j,
// then the digits of the three rows.  fd: [3N][ND][M][M] BF16 (block type
// b = 0: A_j, 1: B_j, 2: -C_j), element (j, b, p, m, k) at
// (((3j + b) ND + p) M + m) M + k.  ea: [N][M].
__global__ void k_fac_digits(const double* __restrict__ A, const double* __restrict__ B,
                             const double* __restrict__ C, int64_t N, int M, __nv_bfloat16* __restrict__ fd,
                             int* __restrict__ ea) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (w >= N * M) return;
  const int64_t j = w / M;
  const int m = (int)(w % M);
  const size_t row = ((size_t)j * M + m) * M;
  unsigned long long mx = 0;
  for (int k = lane; k < M; k += 32) {
    mx = max(mx, (unsigned long long)__double_as_longlong(A[row + k]) & 0x7FFFFFFFFFFFFFFFull);
    mx = max(mx, (unsigned long long)__double_as_longlong(B[row + k]) & 0x7FFFFFFFFFFFFFFFull);
    mx = max(mx, (unsigned long long)__double_as_longlong(C[row + k]) & 0x7FFFFFFFFFFFFFFFull);
  }
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  const int e = scale_of(mx);
  if (lane == 0) ea[w] = e;
  const size_t MM = (size_t)M * M;
  for (int b = 0; b < 3; ++b) {
    const double* src = b == 0 ? A : b == 1 ? B : C;
    for (int k = lane; k < M; k += 32) {
      int d[ND];
      const double v = e == kBadScale ? 0.0 : (b == 2 ? -src[row + k] : src[row + k]);
      digits(v, e == kBadScale ? 0 : e, d);
#pragma unroll
      for (int p = 0; p < ND; ++p)
        fd[((size_t)(3 * j + b) * ND + p) * MM + (size_t)m * M + k] = __float2bfloat16_rn((float)d[p]);
    }
  }
}

__global__ void k_zero_u32(unsigned* p, int64_t n, const int* done) {
  if (done != nullptr && *(volatile const int*)done != 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0u;
}

// Largest |X| of every column over the N*M rows, as the high word of its bit
// pattern with the sign cleared (the exponent field is all the scale needs):
// lanes on consecutive columns, the 8 warps of a CTA and the CTAs of grid.y on
// interleaved rows, four loads in flight per lane, one atomic per column and
// CTA.  32-bit integer maxima only (64-bit ones occupy the FP64 pipe).
__global__ void __launch_bounds__(256) k_colmax(const double* __restrict__ X, int64_t rows, int64_t K,
                                                unsigned* __restrict__ cm, const int* done) {
  if (done != nullptr && *(volatile const int*)done != 0) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * 32 + lane;
  const unsigned* xh = reinterpret_cast<const unsigned*>(X) + 1;  // high words
  unsigned mx = 0;
  if (col < K) {
    const int64_t stride = (int64_t)gridDim.y * 8;
    int64_t r = (int64_t)blockIdx.y * 8 + w;
    for (; r + 3 * stride < rows; r += 4 * stride) {
      const unsigned a = __ldg(xh + 2 * (r * K + col)), b = __ldg(xh + 2 * ((r + stride) * K + col));
      const unsigned c = __ldg(xh + 2 * ((r + 2 * stride) * K + col)), d = __ldg(xh + 2 * ((r + 3 * stride) * K + col));
      mx = max(mx, max(max(a & 0x7FFFFFFFu, b & 0x7FFFFFFFu), max(c & 0x7FFFFFFFu, d & 0x7FFFFFFFu)));
    }
    for (; r < rows; r += stride) mx = max(mx, __ldg(xh + 2 * (r * K + col)) & 0x7FFFFFFFu);
  }
  __shared__ unsigned s[8][32];
  s[w][lane] = mx;
  __syncthreads();
  if (w == 0 && col < K) {
    for (int i = 1; i < 8; ++i) mx = max(mx, s[i][lane]);
    if (mx) atomicMax(cm + col, mx);
  }
}

// X digits, block-transposed: element (p, j, n, k) at ((p N + j) Kp + n) M + k
// (a 128-column tile of block row j is a K-major 128 x M operand); columns
// K..Kp-1 are zero.  A CTA step takes CB = 2048 / M columns of one block row:
// its 256 threads each convert 8 rows of one column, the digits are gathered
// in shared memory and every plane leaves as one contiguous CB * M * 2-byte
// span (whole lines, no partial-sector writes); CTAs stride over the steps.
// e_X(n) to ex[n].
template <int M>
__global__ void __launch_bounds__(256) k_x_digits(const double* __restrict__ X, int64_t N, int64_t K, int64_t Kp,
                                                  const unsigned* __restrict__ cm,
                                                  __nv_bfloat16* __restrict__ xd, int* __restrict__ ex,
                                                  const int* done) {
  if (done != nullptr && *(volatile const int*)done != 0) return;
  constexpr int CB = 2048 / M;  // columns per CTA (x 8-row groups = 256 threads)
  constexpr int RU = M / 8;      // 16-byte units of one column's row of one plane
  // unit (column c, row group kg) of a plane at c * RU + (kg ^ (c & 7)): the
  // eight columns that one store phase of a warp covers hit distinct banks
  __shared__ __align__(16) uint4 sd[ND][CB * RU];
  const int64_t nblk = Kp / CB;
  const int c = threadIdx.x % CB, kg = threadIdx.x / CB;
  const size_t plane = (size_t)N * Kp * M;
  for (int64_t b = blockIdx.x; b < N * nblk; b += gridDim.x) {
    const int64_t j = b / nblk;
    const int64_t n0 = (b % nblk) * CB;
    const int64_t n = n0 + c;
    const int e = n < K ? scale_of((unsigned long long)cm[n] << 32) : 0;
    const bool zero = n >= K || e == kBadScale;
    if (j == 0 && kg == 0) ex[n] = e;
    const double* src = X + ((size_t)j * M + kg * 8) * K + n;
    double v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = zero ? 0.0 : __ldg(src + (size_t)i * K);
    uint32_t w[ND][4];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      int d0[ND], d1[ND];
      digits(v[i], zero ? 0 : e, d0);
      digits(v[i + 1], zero ? 0 : e, d1);
#pragma unroll
      for (int p = 0; p < ND; ++p) w[p][i / 2] = bf2(d0[p], d1[p]);
    }
    __syncthreads();  // the previous span has left shared memory
#pragma unroll
    for (int p = 0; p < ND; ++p) sd[p][c * RU + (kg ^ (c & 7))] = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    __syncthreads();
#pragma unroll
    for (int p = 0; p < ND; ++p) {
      uint4* dst = reinterpret_cast<uint4*>(xd + p * plane + ((size_t)j * Kp + n0) * M);
      for (int u = threadIdx.x; u < CB * RU; u += 256) {
        const int cc = u / RU, kk = u % RU;
        dst[u] = sd[p][cc * RU + (kk ^ (cc & 7))];
      }
    }
  }
}

// --------------------------------------------------------------- outputs
// 8 consecutive rows m of one column, into the block-transposed panel planes
// (plane 1 holds the remainder of the rounding into plane 0).
__device__ __forceinline__ void store8(__nv_bfloat16* o, const float* v, int sp, size_t plane) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    h[i] = *reinterpret_cast<const uint32_t*>(&b);
    const float2 f = __bfloat1622float2(b);
    const __nv_bfloat162 c = __floats2bfloat162_rn(v[2 * i] - f.x, v[2 * i + 1] - f.y);
    l[i] = *reinterpret_cast<const uint32_t*>(&c);
  }
  *reinterpret_cast<uint4*>(o) = make_uint4(h[0], h[1], h[2], h[3]);
  if (sp == 2) *reinterpret_cast<uint4*>(o + plane) = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void store8(float* o, const float* v, int sp, size_t plane) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    float h[4], l[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      h[c] = sp == 2 ? __uint_as_float(__float_as_uint(v[4 * i + c]) & 0xFFFFE000u) : v[4 * i + c];
      l[c] = v[4 * i + c] - h[c];
    }
    reinterpret_cast<float4*>(o)[i] = make_float4(h[0], h[1], h[2], h[3]);
    if (sp == 2) reinterpret_cast<float4*>(o + plane)[i] = make_float4(l[0], l[1], l[2], l[3]);
  }
}

// --------------------------------------------------------------- main kernel
// Output modes: OUT_PANEL -- the tensor-core solve's block-transposed panel
// (TR planes, leading dimension Kp, zero beyond K); OUT_ROWS -- row-major TR
// (leading dimension K); OUT_F64 -- row-major FP64 (diagnostics).
enum { OUT_PANEL = 0, OUT_ROWS = 1, OUT_F64 = 2 };

// Items (block row j, 128-column tile, 64-row half h of the output block),
// the tiles of a block row consecutive: the CTAs at work at one time share the
// factor digit slices of their block rows and the X-digit tiles of
// neighbouring block rows in L2, so each is read from HBM about once.  Per item: for each of the (up to) three
// blocks and each 64-value contraction chunk, the 7 factor digit slices (one
// 4-D TMA box) and the 7 X-digit tiles; 40 MMAs per chunk.
template <int M, int OUT, typename TR>
__global__ void __launch_bounds__(THREADS, 1)
    k_resid_digits(const __grid_constant__ CUtensorMap tm_f, const __grid_constant__ CUtensorMap tm_x,
                   const double* __restrict__ F, const int* __restrict__ ea, const int* __restrict__ ex,
                   void* __restrict__ out, int N, int64_t K, int Kp, int sp, const int* done, double* rn2,
                   const int* cur, int* status) {
  if (done != nullptr && *(volatile const int*)done != 0) return;
  constexpr int MH = M / 64;  // 64-row output halves of a block row
  constexpr int KB = M / 64;  // 64-value contraction chunks of a block
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* sF = sm;             // two factor stacks (7 slices each)
  uint8_t* sX = sm + 2 * FST;   // X-digit tile ring
  uint64_t* bars = reinterpret_cast<uint64_t*>(sX + NX * XT);
  uint64_t* fullF = bars;
  uint64_t* emptyF = bars + 2;
  uint64_t* fullX = bars + 4;
  uint64_t* emptyX = fullX + NX;
  uint64_t* accFull = emptyX + NX;
  uint64_t* accEmpty = accFull + 1;
  uint64_t* drain = accEmpty + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  __shared__ double red[THREADS / 32];

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tiles = Kp / 128;
  const int64_t items = (int64_t)N * tiles * MH;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&fullF[i], 1);
      mbar_init(&emptyF[i], 1);
    }
    for (int i = 0; i < NX; ++i) {
      mbar_init(&fullX[i], 1);
      mbar_init(&emptyX[i], 1);
    }
    mbar_init(accFull, 1);
    mbar_init(accEmpty, 4 * EGW);
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  double part = 0.0;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tm_f);
      prefetch_tmap(&tm_x);
      uint32_t fi = 0, xi = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int h = (int)(it % MH);
        const int64_t t = it / MH;
        const int tile = (int)(t % tiles), j = (int)(t / tiles);
        for (int b = 0; b < 3 && ok; ++b) {
          if ((b == 0 && j == 0) || (b == 1 && j == N - 1)) continue;
          const int jx = b == 0 ? j - 1 : b == 1 ? j + 1 : j;
          for (int kb = 0; kb < KB && ok; ++kb) {
            const uint32_t fs = fi & 1, fu = fi >> 1;
            if (fu > 0 && !mbar_wait(&emptyF[fs], (fu - 1) & 1)) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&fullF[fs], FST);
            tma_load_4d(sF + fs * FST, &tm_f, kb * 64, h * 64, 0, 3 * j + b, &fullF[fs]);
            ++fi;
            for (int q = 0; q < ND; ++q) {
              const uint32_t xs = xi % NX, xu = xi / NX;
              if (xu > 0 && !mbar_wait(&emptyX[xs], (xu - 1) & 1)) {
                ok = false;
                break;
              }
              mbar_arrive_expect_tx(&fullX[xs], XT);
              tma_load_2d(sX + xs * XT, &tm_x, kb * 64, (q * N + jx) * Kp + tile * 128, &fullX[xs]);
              ++xi;
            }
          }
        }
      }
      if (!ok) atomicExch(status, 7);
      // no exit with copies in flight
      for (uint32_t q = 0; q < 2 && q < fi; ++q) {
        const uint32_t l = fi - 1 - q;
        mbar_wait(&fullF[l & 1], (l >> 1) & 1);
      }
      for (uint32_t q = 0; q < NX && q < xi; ++q) {
        const uint32_t l = xi - 1 - q;
        mbar_wait(&fullX[l % NX], (l / NX) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t fi = 0, xi = 0, n = 0;
      bool ok = true;
      // descriptors of the ring bases; a tile or slice at byte offset o is base + o / 16
      const uint64_t xdesc0 = smem_desc(smem_u32(sX), 16, 1024);
      const uint64_t fdesc0 = smem_desc(smem_u32(sF), 16, 1024);
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x, ++n) {
        const int j = (int)(it / MH / tiles);
        if (n > 0 && !mbar_wait(accEmpty, (n - 1) & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        bool first = true;
        for (int b = 0; b < 3 && ok; ++b) {
          if ((b == 0 && j == 0) || (b == 1 && j == N - 1)) continue;
          for (int kb = 0; kb < KB && ok; ++kb) {
            const uint32_t fs = fi & 1;
            if (!mbar_wait(&fullF[fs], (fi >> 1) & 1)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t fd = fdesc0 + (uint64_t)((fs * FST) >> 4);
            // fully unrolled: every instruction's shape (N = 64 np) is a constant
#pragma unroll
            for (int q = 0; q < ND; ++q) {
              if (!ok) break;
              const uint32_t xs = xi % NX;
              if (!mbar_wait(&fullX[xs], (xi / NX) & 1)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint64_t xd = xdesc0 + (uint64_t)((xs * XT) >> 4);
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                // slices p = 0 .. 6 - q, at most four per instruction (16-element K steps: 32 bytes)
#pragma unroll
                for (int p0 = 0; p0 < ND - q; p0 += 4) {
                  const int np = min(4, ND - q - p0);
                  mma_f16(tmem + ACC * (q + p0), xd + 2 * ks, fd + (uint64_t)((p0 * FSL) >> 4) + 2 * ks,
                          instr_desc(1, 0, 128, 64 * np), (first && q == 0 && ks == 0) ? 0u : 1u);
                }
              }
              mma_commit(&emptyX[xs]);
              ++xi;
            }
            mma_commit(&emptyF[fs]);
            ++fi;
            first = false;
          }
        }
        if (ok) mma_commit(accFull);
      }
      if (!ok) atomicExch(status, 8);
      mma_commit(drain);
      mbar_wait(drain, 0);
    }
  } else {
    const int qd = warp & 3, g = (warp - 2) >> 2;  // lane quarter, row group
    const uint32_t lane_base = (uint32_t)(32 * qd) << 16;
    const size_t plane = (size_t)N * Kp * M;
    uint32_t n = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x, ++n) {
      const int h = (int)(it % MH);
      const int64_t t = it / MH;
      const int tile = (int)(t % tiles), j = (int)(t / tiles);
      const int64_t col = (int64_t)tile * 128 + 32 * qd + lane;
      const int m0 = h * 64 + g * RPT;
      const bool colok = col < K;
      const double* Fc = F + ((size_t)j * M + m0) * K + col;  // this thread's RPT rows, stride K
      if (ok) ok = mbar_wait(accFull, n & 1);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
      if (!ok) break;
      tc_fence_after();
      // phase 1: drain the 7 accumulators of this thread's RPT rows into T (int64,
      // modulo 2^64) and Th ~ T / 2^35 (FP32, from the two leading sums)
      uint64_t T[RPT];
      float Th[RPT];
#pragma unroll
      for (int c = 0; c < RPT / 8; ++c) {
        const uint32_t a = tmem + lane_base + g * RPT + c * 8;
        uint32_t r0[32], r1[24];
        tmem_ld8x4(a, a + ACC, a + 2 * ACC, a + 3 * ACC, r0);
        tmem_ld8x3(a + 4 * ACC, a + 5 * ACC, a + 6 * ACC, r1);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float v0 = __uint_as_float(r0[i]), v1 = __uint_as_float(r0[8 + i]);
          // every sum is below 2^24, so each pair c_d 128 + c_{d+1} fits in 31 bits
          const int p01 = __float2int_rn(v0) * 128 + __float2int_rn(v1);
          const int p23 = __float2int_rn(__uint_as_float(r0[16 + i])) * 128 + __float2int_rn(__uint_as_float(r0[24 + i]));
          const int p45 = __float2int_rn(__uint_as_float(r1[i])) * 128 + __float2int_rn(__uint_as_float(r1[8 + i]));
          const int c6 = __float2int_rn(__uint_as_float(r1[16 + i]));
          uint64_t tt = (uint64_t)(int64_t)p01 * 16384u + (uint64_t)(int64_t)p23;
          tt = tt * 16384u + (uint64_t)(int64_t)p45;
          T[8 * c + i] = tt * 128u + (uint64_t)(int64_t)c6;
          Th[8 * c + i] = fmaf(v0, 128.f, v1);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(accEmpty);
      // phase 2 (overlaps the next item's MMAs): add F, round, store, in chunks
      // of 8 rows, the next chunk of F in flight meanwhile
      const int e_x = ex[col];
      const int* ear = ea + (size_t)j * M + m0;
      int eam = -100000;
#pragma unroll
      for (int i = 0; i < RPT; ++i) eam = max(eam, __ldg(ear + i));
      float nf = 0.f;
      double nbig = 0.0;
#pragma unroll
      for (int c = 0; c < RPT / 8; ++c) {
        double Fv[8];
        int eav[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          Fv[i] = colok ? __ldg(Fc + (size_t)(8 * c + i) * K) : 0.0;
          eav[i] = __ldg(ear + 8 * c + i);
        }
        float rs[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int ii = 8 * c + i;
          const size_t orow = ((size_t)j * M + m0 + ii) * K + col;
          const int E = eav[i] + e_x;
          // F = (-1)^neg mant 2^(be' - 1075), be' = max(be, 1)
          const uint64_t fb = (uint64_t)__double_as_longlong(Fv[i]);
          const int be = (int)((fb >> 52) & 0x7FF);
          const uint64_t mant = (fb & 0xFFFFFFFFFFFFFull) | (be ? (1ull << 52) : 0ull);
          const int eu = be - 1023 - (E - 56) - 35;  // exponent of F / (u 2^35)
          // FP32 estimate of r / (u 2^35) (its error is far below the 2^27 threshold)
          const float ff = (be == 0 || eu < -126)
                               ? 0.f
                               : __int_as_float((int)(((uint32_t)(fb >> 63) << 31) | ((uint32_t)(eu + 127) << 23) |
                                                      (uint32_t)((mant >> 29) & 0x7FFFFFu)));
          const bool slow = e_x == kBadScale || eav[i] == kBadScale || be == 0x7FF || eu > 47 ||
                            !(fabsf(ff + Th[ii]) < 0x1p27f);
          double rd = 0.0;
          float r;
          if (!slow) {
            // F / u to the unit below (truncated), modulo 2^64
            const int sh = max(be, 1) - 1075 - (E - 56);
            uint64_t ffix = sh >= 0 ? shl64(mant, (uint32_t)sh) : shr64(mant, (uint32_t)(-sh));
            if (fb >> 63) ffix = 0ull - ffix;
            const int64_t R = (int64_t)(ffix + T[ii]);
            const float rf = __ll2float_rn(R);
            const int es = E - 56;
            r = ((unsigned)(es + 126) <= 253u) ? rf * pow2f(es) : scale_f(rf, es);
            const int en = eav[i] - eam - 56;
            const float un = en >= -126 ? rf * pow2f(en) : 0.f;
            nf = fmaf(un, un, nf);
            if constexpr (OUT == OUT_F64) rd = ldexp(__ll2double_rn(R), es);
          } else if (e_x == kBadScale || eav[i] == kBadScale) {
            r = __int_as_float(0x7FC00000);
            rd = __longlong_as_double(0x7FF8000000000000ll);
            nbig = rd;
          } else {
            // r far from cancellation, or F non-finite: FP64, with the exact T
            // recovered from its estimate (|T - Th 2^35| < 2^53, far below 2^64)
            const double Ts = (double)(int64_t)T[ii];
            const double kk = rint(((double)Th[ii] * 0x1p35 - Ts) * 0x1p-64);
            rd = ldexp(Ts + kk * 0x1p64, E - 56) + Fv[i];
            r = (float)rd;
            nbig = fma(rd, rd, nbig);
          }
          rs[i] = r;
          if constexpr (OUT == OUT_F64) {
            if (colok) reinterpret_cast<double*>(out)[orow] = rd;
          } else if constexpr (OUT == OUT_ROWS) {
            if (colok) reinterpret_cast<TR*>(out)[orow] = (TR)r;
          }
        }
        if constexpr (OUT == OUT_PANEL)
          store8(reinterpret_cast<TR*>(out) + ((size_t)j * Kp + col) * M + m0 + 8 * c, rs, sp, plane);
      }
      if (colok) part += ldexp((double)nf, 2 * (eam + e_x)) + nbig;
    }
    if (!ok && lane == 0) atomicExch(status, 9);
  }
  // the squared norm: one atomic per CTA
  for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
  if (lane == 0) red[warp] = part;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0 && rn2 != nullptr) {
    double s = 0.0;
    for (int w = 0; w < THREADS / 32; ++w) s += red[w];
    if (s != 0.0 || s != s) atomicAdd(rn2 + (cur ? *cur : 0), s);
  }
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// --------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bt_status encode_bf16(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                      const cuuint32_t* box) {
  auto enc = tmap_encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return BT_ERR_CUDA;
  }
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return BT_ERR_CUDA;
  }
  return BT_OK;
}

bt_status grow_buf(bt_handle_s* h, void** p, size_t* have, size_t need, cudaStream_t s) {
  if (need <= *have) return BT_OK;
  if (*p) {
    BT_CUDA(cudaStreamSynchronize(s));
    BT_CUDA(cudaFree(*p));
    *p = nullptr;
    *have = 0;
  }
  const cudaError_t e = cudaMalloc(p, need);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error(std::string("residual buffer allocation failed: ") + cudaGetErrorString(e));
    return BT_ERR_OOM;
  }
  *have = need;
  ++h->lp_gen;  // captured graphs hold the old pointers
  return BT_OK;
}

template <int M, int OUT, typename TR>
bt_status launch_main(const CUtensorMap& tf, const CUtensorMap& tx, const double* F, const int* ea, const int* ex,
                      void* out, int N, int64_t K, int Kp, int sp, const int* done, double* rn2, const int* cur,
                      int* status, cudaStream_t s) {
  auto kern = k_resid_digits<M, OUT, TR>;
  BT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
  int sms = 0, dev = 0;
  BT_CUDA(cudaGetDevice(&dev));
  BT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t items = (int64_t)N * (Kp / 128) * (M / 64);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, sms));
  kern<<<grid, THREADS, SMEM, s>>>(tf, tx, F, ea, ex, out, N, K, Kp, sp, done, rn2, cur, status);
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

}  // namespace

bool resid_digits_supported(const bt_handle_s* h, int64_t K) {
  const int64_t Kp = (K + 127) / 128 * 128;
  return !h->stencil && (h->M == 64 || h->M == 128) && K >= 1 && (int64_t)ND * h->N * Kp < (int64_t)1 << 31 &&
         3 * h->N < ((int64_t)1 << 31);
}

bt_status resid_digits_prepare(bt_handle_s* h, int64_t K, cudaStream_t s) {
  const int64_t N = h->N, M = h->M, Kp = (K + 127) / 128 * 128;
  if (!h->dg_fac) {
    void* fd = nullptr;
    void* e = nullptr;
    size_t have = 0, have2 = 0;
    BT_TRY(grow_buf(h, &fd, &have, (size_t)3 * N * ND * M * M * sizeof(__nv_bfloat16), s));
    const bt_status st2 = grow_buf(h, &e, &have2, (size_t)N * M * sizeof(int), s);
    if (st2 != BT_OK) {
      cudaFree(fd);
      return st2;
    }
    const int64_t warps = N * M;
    k_fac_digits<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(h->A, h->B, h->C, N, (int)M,
                                                             reinterpret_cast<__nv_bfloat16*>(fd),
                                                             reinterpret_cast<int*>(e));
    BT_CUDA(cudaGetLastError());
    h->dg_fac = fd;
    h->dg_ea = reinterpret_cast<int*>(e);
  }
  BT_TRY(grow_buf(h, &h->dg_x, &h->dg_x_bytes, (size_t)ND * N * Kp * M * sizeof(__nv_bfloat16), s));
  BT_TRY(grow_buf(h, &h->dg_col, &h->dg_col_bytes, (size_t)Kp * (sizeof(unsigned) + sizeof(int)), s));
  return BT_OK;
}

// out_mode 0: the tensor-core panel (TR = float if tr_float, else BF16; sp
// planes, leading dimension Kp = K rounded up to 128); 1: row-major FP32
// (leading dimension K); 2: row-major FP64.  rn2[*cur] (rn2[0] without cur)
// receives the squared norm.  resid_digits_prepare must have run for K.
bt_status launch_resid_digits(bt_handle_s* h, const double* F, const double* X, int64_t K, int out_mode,
                              bool tr_float, void* out, int sp, const int* done, double* rn2, const int* cur,
                              int* status, cudaStream_t s) {
  const int64_t N = h->N, M = h->M, Kp = (K + 127) / 128 * 128;
  unsigned* cm = reinterpret_cast<unsigned*>(h->dg_col);
  int* ex = reinterpret_cast<int*>(cm + Kp);
  __nv_bfloat16* xd = reinterpret_cast<__nv_bfloat16*>(h->dg_x);
  {
    ProfScope ps(h, s, "resid_prep");
    k_zero_u32<<<(unsigned)std::min<int64_t>((Kp + 255) / 256, 1024), 256, 0, s>>>(cm, Kp, done);
    const int64_t rows = N * M;
    const unsigned gx = (unsigned)((K + 31) / 32);
    const unsigned gy =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, std::max<int64_t>(1, 1216 / (int64_t)gx)));
    k_colmax<<<dim3(gx, gy), 256, 0, s>>>(X, rows, K, cm, done);
    if (M == 64) {
      static const int grid = resident_grid(reinterpret_cast<const void*>(&k_x_digits<64>), 256, 0);
      k_x_digits<64><<<(unsigned)std::min<int64_t>(N * (Kp / 32), grid), 256, 0, s>>>(X, N, K, Kp, cm, xd, ex, done);
    } else {
      static const int grid = resident_grid(reinterpret_cast<const void*>(&k_x_digits<128>), 256, 0);
      k_x_digits<128><<<(unsigned)std::min<int64_t>(N * (Kp / 16), grid), 256, 0, s>>>(X, N, K, Kp, cm, xd, ex, done);
    }
    BT_CUDA(cudaGetLastError());
  }
  CUtensorMap tf, tx;
  {
    const cuuint64_t dims[4] = {(cuuint64_t)M, (cuuint64_t)M, (cuuint64_t)ND, (cuuint64_t)(3 * N)};
    const cuuint64_t strides[3] = {(cuuint64_t)M * 2, (cuuint64_t)M * M * 2, (cuuint64_t)ND * M * M * 2};
    const cuuint32_t box[4] = {64, 64, (cuuint32_t)ND, 1};
    BT_TRY(encode_bf16(&tf, h->dg_fac, 4, dims, strides, box));
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)(ND * N * Kp)};
    const cuuint64_t strides[1] = {(cuuint64_t)M * 2};
    const cuuint32_t box[2] = {64, 128};
    BT_TRY(encode_bf16(&tx, xd, 2, dims, strides, box));
  }
  ProfScope ps(h, s, "residual");
  const int n = (int)N, kp = (int)Kp;
  if (M == 64) {
    if (out_mode == OUT_PANEL && !tr_float)
      return launch_main<64, OUT_PANEL, __nv_bfloat16>(tf, tx, F, h->dg_ea, ex, out, n, K, kp, sp, done, rn2, cur,
                                                        status, s);
    if (out_mode == OUT_PANEL)
      return launch_main<64, OUT_PANEL, float>(tf, tx, F, h->dg_ea, ex, out, n, K, kp, sp, done, rn2, cur, status, s);
    if (out_mode == OUT_ROWS)
      return launch_main<64, OUT_ROWS, float>(tf, tx, F, h->dg_ea, ex, out, n, K, kp, sp, done, rn2, cur, status, s);
    return launch_main<64, OUT_F64, float>(tf, tx, F, h->dg_ea, ex, out, n, K, kp, sp, done, rn2, cur, status, s);
  }
  if (out_mode == OUT_PANEL && !tr_float)
    return launch_main<128, OUT_PANEL, __nv_bfloat16>(tf, tx, F, h->dg_ea, ex, out, n, K, kp, sp, done, rn2, cur,
                                                       status, s);
  if (out_mode == OUT_PANEL)
    return launch_main<128, OUT_PANEL, float>(tf, tx, F, h->dg_ea, ex, out, n, K, kp, sp, done, rn2, cur, status, s);
  if (out_mode == OUT_ROWS)
    return launch_main<128, OUT_ROWS, float>(tf, tx, F, h->dg_ea, ex, out, n, K, kp, sp, done, rn2, cur, status, s);
  return launch_main<128, OUT_F64, float>(tf, tx, F, h->dg_ea, ex, out, n, K, kp, sp, done, rn2, cur, status, s);
}

}  // namespace bt
