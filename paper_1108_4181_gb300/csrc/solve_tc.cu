// Algorithm 2, stage 2 on the tcgen05 tensor cores (BF16 or TF32 operands,
// FP32 accumulation in TMEM), used as the inner solve of iterative refinement.
//
// Internal panels (residual r, work panel holding y, W, F~ and X~) are stored
// block-transposed: block row j of a panel is a K x M matrix, element (m, n)
// at (j * Kp + n) * M + m, Kp = K rounded up to 128.  A column tile of a
// block row is then an NT x M matrix with M contiguous, and a factor block
// (row-major M x M) is M rows with M contiguous: both are K-major operands
// for BF16 and TF32, moved by TMA with 128-byte swizzle.
//
// Operand roles.  The default roles put the factor block in the MMA's A
// operand (M rows) and the panel tile in B (NT columns).  The swapped roles
// (Cfg SW, used for the split-BF16 precision) put the 128-column panel tile
// in A and the factor block in B (N = M), so every MMA is 128 x M x 16 and
// the accumulator holds the transposed product: TMEM lane = panel column,
// one epilogue thread owns a contiguous column of the result.
//
// Split operands (SP = 2): every factor and panel value v is stored as two
// planes hi = round(v), lo = round(v - hi), and each product is formed as
// hi*hi + hi*lo + lo*hi (three MMAs, FP32 accumulation), which carries
// about twice the operand precision (BF16: ~2^-17 instead of 2^-9) and cuts
// the number of refinement passes.
//
//   k_tc_sweep       eq. sub3 per (segment, column tile), step 2.1:
//                    forward  y_i = Dinv_i r_i + E_i y_{i-1} (with A_i = I:
//                    Dinv_i (r_i + y_{i-1}) from the same Dinv slices),
//                    backward W_i = y_i + G_i W_{i+1}.  Warp 0 streams factor
//                    slices and panel tiles with TMA into rings, warp 1 issues
//                    the MMAs (one thread), warps 2-9 drain the TMEM
//                    accumulator, write the next recurrence operand into
//                    shared memory and store the row with TMA.  Two
//                    accumulators let the next row's MMAs start while the
//                    previous row is drained.
//   k_tc_ifgemm      step 2.2 (split BF16): jobs of up to two block products
//                    plus an add -- F~ (eq. red1), the series terms R F~, and
//                    one launch per dichotomy level (Algorithm 1) -- with the
//                    node sums of the series terms from k_node_sums.
//   k_tc_iface / k_tc_dichotomy   step 2.2 on the CUDA cores in FP32 for the
//                    single-plane precisions.
//   k_tc_correct_ta  eq. superposition, step 2.3 (split BF16, M = 128):
//                    d_i = W_i + U_i X~_s + V_i X~_{s+1} with the two
//                    interface tiles as TMEM A operands; k_tc_correct for the
//                    other configurations.  d goes to an FP32 panel.
//   k_x_update_warp  X (+)= d into the caller's FP64 solution.

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <cstdlib>
#include <cstring>

#include "bt_internal.cuh"
#include "fpconv.cuh"
#include "tc_ptx.cuh"

namespace bt {

namespace {

using namespace tc;

// ------------------------------------------------------------------ traits
template <typename E>
struct ET;
template <>
struct ET<__nv_bfloat16> {
  static constexpr uint32_t fmt = 1;
  static constexpr CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  static __device__ __forceinline__ float tof(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
  // v = hi + lo with hi, lo representable
  static __device__ __forceinline__ void split(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
};
template <>
struct ET<float> {
  static constexpr uint32_t fmt = 2;
  static constexpr CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  static __device__ __forceinline__ float tof(float v) { return v; }
  static __device__ __forceinline__ float from(float v) { return v; }
  static __device__ __forceinline__ void split(float v, float& hi, float& lo) {
    hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);  // exactly a TF32 value
    lo = v - hi;
  }
};

__host__ __device__ constexpr int pow2ceil(int v) {
  int p = 32;
  while (p < v) p *= 2;
  return p;
}

// SW_ (swapped operand roles): the panel tile is the MMA's A operand (NT = 128
// rows: the tile's columns n) and the factor block the B operand (N = M: its
// rows); the accumulator then holds the transposed product -- TMEM lane n,
// column m' -- and one epilogue thread owns a whole column of the result, so
// it reads and writes the K-major panel tiles in 16-byte vectors.  Both
// operands keep the K-major 128-byte-swizzled smem layout of the default
// roles (factor slice: rows x 128 B; panel tile: NT rows x 128 B per chunk).
template <typename E, int M_, int NT_, int NA_, int SP_, int NP_ = 2, bool SW_ = false, int EG_ = 2>
struct Cfg {
  static constexpr int M = M_, NT = NT_, NA = NA_, SP = SP_, NP = NP_;  // NP: panel-ring stages
  static constexpr bool SW = SW_;
  static constexpr int eb = (int)sizeof(E);
  static constexpr int CE = 128 / eb;      // elements in one 128-byte swizzle row
  static constexpr int KS = 32 / eb;       // K of one MMA instruction
  static constexpr int NCH = M / CE;       // 128-byte chunks per block row / per tile row
  static constexpr int SLICE = M * 128;    // one A slice of one plane: M rows x 128 bytes
  static constexpr int SLOT = SP * SLICE;  // one ring slot: the slice of every plane
  static constexpr int TCH = NT * 128;     // one tile chunk: NT rows x 128 bytes
  static constexpr int TILE = NCH * TCH;   // one NT x M panel tile of one plane
  static constexpr int PT = SP * TILE;     // a panel tile with all its planes
  static constexpr int ACC = SW ? M : NT;         // TMEM columns of one accumulator buffer
  static constexpr int TMEM_COLS = pow2ceil(2 * ACC);
  static constexpr uint32_t IDESC = SW ? instr_desc(ET<E>::fmt, 0, NT, M) : instr_desc(ET<E>::fmt, 0, M, NT);
  static constexpr int EG = EG_;                // epilogue warp groups, each drains ACC/EG columns
  static constexpr int NH = NT / EG;            // default roles: tile columns per epilogue thread
  static constexpr int MH = M / EG;             // swapped roles: block rows per epilogue thread
  static constexpr int YB = SW ? 1 : 2;         // recurrence-operand buffers of the sweep
  static constexpr int THREADS = 64 + 128 * EG;
  static_assert(NH % 16 == 0, "epilogue column share");
  static_assert(!SW || (NT == 128 && MH % 32 == 0), "swapped roles: 128-column tiles");
  static_assert(M == 64 || M == 128, "tensor-core path supports M = 64 and M = 128");
  static_assert(NT % 32 == 0 && NT <= 256, "column tile");
  static_assert(TCH % 1024 == 0, "swizzle atoms");
  static_assert(SP == 1 || SP == 2, "one or two planes");
};

// Byte offset of element (n, m) inside a K-major 128B-swizzled NT x M tile.
template <class C>
__device__ __forceinline__ uint32_t kmaj_off(int n, int m) {
  constexpr int per16 = 16 / C::eb;
  const int c = m / C::CE;
  const int u = (m % C::CE) / per16;
  return (uint32_t)(c * C::TCH + n * 128 + ((u ^ (n & 7)) << 4) + (m % per16) * C::eb);
}

// Value (n, m) of a panel tile with all its planes.
template <typename E, class C>
__device__ __forceinline__ float tile_get(const uint8_t* tile, int n, int m) {
  const uint32_t o = kmaj_off<C>(n, m);
  float v = ET<E>::tof(*reinterpret_cast<const E*>(tile + o));
  if (C::SP == 2) v += ET<E>::tof(*reinterpret_cast<const E*>(tile + C::TILE + o));
  return v;
}

template <typename E, class C>
__device__ __forceinline__ void tile_put(uint8_t* tile, int n, int m, float v) {
  const uint32_t o = kmaj_off<C>(n, m);
  if (C::SP == 2) {
    E hi, lo;
    ET<E>::split(v, hi, lo);
    *reinterpret_cast<E*>(tile + o) = hi;
    *reinterpret_cast<E*>(tile + C::TILE + o) = lo;
  } else {
    *reinterpret_cast<E*>(tile + o) = ET<E>::from(v);
  }
}

// ---- swapped roles: whole rows (one tile column n, block rows m0..m0+MH) of a
// K-major swizzled tile, 16 bytes at a time.
template <class C>
__device__ __forceinline__ uint32_t unit_off(int n, int m) {
  constexpr int per16 = 16 / C::eb;
  return (uint32_t)((m / C::CE) * C::TCH + n * 128 + ((((m % C::CE) / per16) ^ (n & 7)) << 4));
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }

// 16 bytes of planes 0 (rounded) and 1 (remainder) from per16 FP32 values.
template <typename E, int SP>
__device__ __forceinline__ void pack16(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4] = {0u, 0u, 0u, 0u};
  if constexpr (sizeof(E) == 2) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
      h[q] = bf2_bits(b);
      if (SP == 2) {
        const float2 f = __bfloat1622float2(b);
        l[q] = bf2_bits(__floats2bfloat162_rn(v[2 * q] - f.x, v[2 * q + 1] - f.y));
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (SP == 2) {
        h[q] = __float_as_uint(v[q]) & 0xFFFFE000u;  // exactly a TF32 value
        l[q] = __float_as_uint(v[q] - __uint_as_float(h[q]));
      } else {
        h[q] = __float_as_uint(v[q]);
      }
    }
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// v[j] += value (n, m0 + j) summed over the planes, from 16-byte units.
template <typename E, int SP>
__device__ __forceinline__ void unpack16_add(const uint4& hi, const uint4& lo, float* v) {
  const uint32_t h[4] = {hi.x, hi.y, hi.z, hi.w}, l[4] = {lo.x, lo.y, lo.z, lo.w};
  if constexpr (sizeof(E) == 2) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h[q]));
      if (SP == 2) {
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&l[q]));
        a.x += b.x;
        a.y += b.y;
      }
      v[2 * q] += a.x;
      v[2 * q + 1] += a.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] += __uint_as_float(h[q]) + (SP == 2 ? __uint_as_float(l[q]) : 0.f);
  }
}

template <typename E, class C>
__device__ __forceinline__ void row_put(uint8_t* tile, int n, int m0, const float (&v)[C::MH]) {
  constexpr int per16 = 16 / C::eb;
#pragma unroll
  for (int u = 0; u < C::MH / per16; ++u) {
    uint4 hi, lo;
    pack16<E, C::SP>(&v[u * per16], hi, lo);
    const uint32_t o = unit_off<C>(n, m0 + u * per16);
    *reinterpret_cast<uint4*>(tile + o) = hi;
    if (C::SP == 2) *reinterpret_cast<uint4*>(tile + C::TILE + o) = lo;
  }
}

template <typename E, class C>
__device__ __forceinline__ void row_add(const uint8_t* tile, int n, int m0, float (&v)[C::MH]) {
  constexpr int per16 = 16 / C::eb;
#pragma unroll
  for (int u = 0; u < C::MH / per16; ++u) {
    const uint32_t o = unit_off<C>(n, m0 + u * per16);
    const uint4 hi = *reinterpret_cast<const uint4*>(tile + o);
    const uint4 lo = C::SP == 2 ? *reinterpret_cast<const uint4*>(tile + C::TILE + o) : make_uint4(0, 0, 0, 0);
    unpack16_add<E, C::SP>(hi, lo, &v[u * per16]);
  }
}

// TMEM lane holding accumulator row `row` (cta_group::1): M = 128 uses all 128
// lanes, M = 64 the first 16 lanes of each 32-lane quadrant.
template <class C>
__device__ __forceinline__ void epi_row(int warp, int lane, int* row, bool* has) {
  const int q = warp & 3;
  if (C::M == 128) {
    *row = 32 * q + lane;
    *has = true;
  } else {
    *row = 16 * q + (lane & 15);
    *has = lane < 16;
  }
}

__device__ __forceinline__ bool flag_set(const int* f) { return f != nullptr && *(volatile const int*)f != 0; }

struct Bars {
  uint64_t* fullA;
  uint64_t* emptyA;
  uint64_t* fullP;
  uint64_t* emptyP;
  uint64_t* mdone;
  uint64_t* afree;
  uint64_t* yrdy;
  uint64_t* extra;  // [0] forward stores complete / B tiles loaded, [1] drain
};

template <class C>
__device__ __forceinline__ Bars carve(uint64_t* b) {
  Bars r;
  r.fullA = b;
  r.emptyA = b + C::NA;
  r.fullP = b + 2 * C::NA;
  r.emptyP = r.fullP + C::NP;
  r.mdone = r.emptyP + C::NP;
  r.afree = r.mdone + 2;
  r.yrdy = r.afree + 2;
  r.extra = r.yrdy + 2;
  return r;
}

__host__ __device__ constexpr int kBars(int na, int np) { return 2 * na + 2 * np + 8; }

template <class C>
__device__ __forceinline__ void init_bars(const Bars& b) {
  for (int i = 0; i < C::NA; ++i) {
    mbar_init(&b.fullA[i], 1);
    mbar_init(&b.emptyA[i], 1);
  }
  for (int i = 0; i < C::NP; ++i) {
    mbar_init(&b.fullP[i], 1);
    mbar_init(&b.emptyP[i], 1);
  }
  for (int i = 0; i < 2; ++i) {
    mbar_init(&b.mdone[i], 1);
    mbar_init(&b.afree[i], 4 * C::EG);
    mbar_init(&b.yrdy[i], 1);
    mbar_init(&b.extra[i], 1);
  }
  fence_mbar_init();
}

// Producer helper: one A slice (every plane) into the ring; waits for the slot.
// fplane: tensor-map rows between factor planes.
template <class C>
__device__ __forceinline__ bool load_slice(uint8_t* sA, const Bars& b, uint32_t& ai, const CUtensorMap* tm, int x,
                                           int y, int fplane) {
  const uint32_t slot = ai % C::NA, use = ai / C::NA;
  if (use > 0 && !mbar_wait(&b.emptyA[slot], (use - 1) & 1)) return false;
  mbar_arrive_expect_tx(&b.fullA[slot], C::SLOT);
#pragma unroll
  for (int p = 0; p < C::SP; ++p) tma_load_2d(sA + slot * C::SLOT + p * C::SLICE, tm, x, y + p * fplane, &b.fullA[slot]);
  ++ai;
  return true;
}

// Producer helper: one panel tile (every plane, NCH boxes each) into the P ring.
// pplane: tensor-map rows between panel planes.
template <class C>
__device__ __forceinline__ bool load_tile(uint8_t* sP, const Bars& b, uint32_t& pi, const CUtensorMap* tm, int y,
                                          int pplane) {
  const uint32_t slot = pi % C::NP, use = pi / C::NP;
  if (use > 0 && !mbar_wait(&b.emptyP[slot], (use - 1) & 1)) return false;
  mbar_arrive_expect_tx(&b.fullP[slot], C::PT);
#pragma unroll
  for (int p = 0; p < C::SP; ++p)
    for (int c = 0; c < C::NCH; ++c)
      tma_load_2d(sP + slot * C::PT + p * C::TILE + c * C::TCH, tm, c * C::CE, y + p * pplane, &b.fullP[slot]);
  ++pi;
  return true;
}

template <typename E>
__device__ __forceinline__ void mma1(uint32_t d, uint64_t a, uint64_t bdesc, uint32_t idesc, bool acc) {
  if (ET<E>::fmt == 1)
    mma_f16(d, a, bdesc, idesc, acc ? 1u : 0u);
  else
    mma_tf32(d, a, bdesc, idesc, acc ? 1u : 0u);
}

// MMA helper: D (+)= A_block * B_tile over the M-long contraction, streaming
// the block's NCH slices from the ring; frees each slot when consumed.  With
// two planes: D += Ahi Bhi + Ahi Blo + Alo Bhi.
// The MMAs of one contraction chunk (CE values) of one factor slice (at smem
// address fslot, all planes) against chunk c of a panel tile: D (+)= slice x
// tile (roles per C::SW); with two planes hi*hi + hi*lo + lo*hi.
template <typename E, class C>
__device__ __forceinline__ void mma_chunk(uint32_t dtmem, uint32_t fslot, uint32_t btile, int c, bool& first) {
#pragma unroll
  for (int kq = 0; kq < C::CE / C::KS; ++kq) {
    const uint32_t boff = btile + c * C::TCH + kq * 32;
    const uint64_t fhi = smem_desc(fslot + kq * 32, 16, 1024), phi = smem_desc(boff, 16, 1024);
    if constexpr (C::SW) {
      mma1<E>(dtmem, phi, fhi, C::IDESC, !first);
      first = false;
      if (C::SP == 2) {
        mma1<E>(dtmem, smem_desc(boff + C::TILE, 16, 1024), fhi, C::IDESC, true);
        mma1<E>(dtmem, phi, smem_desc(fslot + C::SLICE + kq * 32, 16, 1024), C::IDESC, true);
      }
    } else {
      mma1<E>(dtmem, fhi, phi, C::IDESC, !first);
      first = false;
      if (C::SP == 2) {
        mma1<E>(dtmem, fhi, smem_desc(boff + C::TILE, 16, 1024), C::IDESC, true);
        mma1<E>(dtmem, smem_desc(fslot + C::SLICE + kq * 32, 16, 1024), phi, C::IDESC, true);
      }
    }
  }
}

// MMA helper: D (+)= A_block * B_tile over the M-long contraction, streaming
// the block's NCH slices from the ring; frees each slot when consumed.
template <typename E, class C>
__device__ __forceinline__ bool mma_block(uint8_t* sA, const Bars& b, uint32_t& ai, uint32_t dtmem, uint32_t btile,
                                          bool& first) {
  for (int c = 0; c < C::NCH; ++c) {
    const uint32_t slot = ai % C::NA, use = ai / C::NA;
    if (!mbar_wait(&b.fullA[slot], use & 1)) return false;
    tc_fence_after();
    mma_chunk<E, C>(dtmem, smem_u32(sA + slot * C::SLOT), btile, c, first);
    mma_commit(&b.emptyA[slot]);
    ++ai;
  }
  return true;
}

// Drains NH accumulator columns of this thread's TMEM lane into v[].
template <int NH>
__device__ __forceinline__ void tmem_cols(uint32_t taddr, float (&v)[NH]) {
  if constexpr (NH % 32 == 0) {
#pragma unroll
    for (int c0 = 0; c0 < NH; c0 += 32) {
      float t[32];
      tmem_ld32(taddr + c0, t);
#pragma unroll
      for (int i = 0; i < 32; ++i) v[c0 + i] = t[i];
    }
  } else {
#pragma unroll
    for (int c0 = 0; c0 < NH; c0 += 16) {
      float t[16];
      tmem_ld16(taddr + c0, t);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[c0 + i] = t[i];
    }
  }
}

// Factor block types in the combined low-precision factor array [SP][5][N][M][M].
enum { FT_DINV = 0, FT_E = 1, FT_G = 2, FT_U = 3, FT_V = 4 };

// ======================================================================
// Sweep kernel
// ======================================================================
template <typename E, class C>
__global__ void __launch_bounds__(C::THREADS, 1)
    k_tc_sweep(const __grid_constant__ CUtensorMap tm_fac, const __grid_constant__ CUtensorMap tm_r,
               const __grid_constant__ CUtensorMap tm_w, int N, int L, int Kp, int shareD,
               const int* done, int* status) {
  if (flag_set(done)) return;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = sm;
  uint8_t* sP = sA + C::NA * C::SLOT;
  uint8_t* sY = sP + C::NP * C::PT;
  uint64_t* barmem = reinterpret_cast<uint64_t*>(sY + C::YB * C::PT);
  const Bars b = carve<C>(barmem);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(barmem + kBars(C::NA, C::NP));

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n0 = blockIdx.x * C::NT;
  const int s = blockIdx.y;
  const int a = s * L + 1;       // first interior row
  const int nrow = L - 1;        // interior rows
  const int T = nrow >= 2 ? 2 * nrow - 1 : nrow;
  const int fplane = 5 * N * C::M;  // tensor-map rows per factor plane
  const int pplane = N * Kp;        // tensor-map rows per panel plane

  if (threadIdx.x == 0) init_bars<C>(b);
  if (warp == 1) {
    tmem_alloc(tslot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tm_fac);
      prefetch_tmap(&tm_r);
      prefetch_tmap(&tm_w);
      uint32_t ai = 0, pi = 0;
      bool ok = true;
      for (int t = 0; t < T && ok; ++t) {
        const bool fwd = t < nrow;
        const int o = fwd ? t : nrow - 2 - (t - nrow);
        const int i = a + o;
        if (!fwd && t == nrow) ok = mbar_wait(&b.extra[0], 0);
        if (ok) ok = load_tile<C>(sP, b, pi, fwd ? &tm_r : &tm_w, i * Kp + n0, pplane);
        const int first_type = fwd ? FT_DINV : FT_G;
        for (int c = 0; c < C::NCH && ok; ++c)
          ok = load_slice<C>(sA, b, ai, &tm_fac, c * C::CE, (first_type * N + i) * C::M, fplane);
        if (fwd && t > 0 && !shareD)
          for (int c = 0; c < C::NCH && ok; ++c)
            ok = load_slice<C>(sA, b, ai, &tm_fac, c * C::CE, (FT_E * N + i) * C::M, fplane);
      }
      if (!ok) atomicExch(status, 1);
      // no copy may still be landing when the CTA exits
      for (uint32_t q = 0; q < C::NA && q < ai; ++q) {
        const uint32_t last = (ai - 1 - q);
        mbar_wait(&b.fullA[last % C::NA], (last / C::NA) & 1);
      }
      for (uint32_t q = 0; q < C::NP && q < pi; ++q) {
        const uint32_t last = pi - 1 - q;
        mbar_wait(&b.fullP[last % C::NP], (last / C::NP) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t ai = 0, pi = 0;
      bool ok = true;
      for (int t = 0; t < T && ok; ++t) {
        const bool fwd = t < nrow;
        const int bsel = t & 1;
        const uint32_t dt = tmem + bsel * C::ACC;
        const uint32_t yop = smem_u32(sY + (C::YB == 2 ? ((t - 1) & 1) : 0) * C::PT);  // y_{t-1} / W_{i+1}
        if (t >= 2) ok = mbar_wait(&b.afree[bsel], ((t >> 1) - 1) & 1);
        tc_fence_after();
        bool first = true;
        uint32_t pslot = 0;
        if (ok && fwd && shareD && t > 0) {
          // A_i = I: E_i = Dinv_i, so y_i = Dinv_i (r_i + y_{i-1}); each Dinv
          // slice serves both products and is released after the second
          pslot = pi % C::NP;
          ok = mbar_wait(&b.fullP[pslot], (pi / C::NP) & 1);
          tc_fence_after();
          const uint32_t ai0 = ai;
          for (int c = 0; c < C::NCH && ok; ++c) {
            const uint32_t q = ai0 + c, slot = q % C::NA;
            ok = mbar_wait(&b.fullA[slot], (q / C::NA) & 1);
            tc_fence_after();
            if (ok) mma_chunk<E, C>(dt, smem_u32(sA + slot * C::SLOT), smem_u32(sP + pslot * C::PT), c, first);
          }
          if (ok) ok = mbar_wait(&b.yrdy[(t - 1) & 1], ((t - 1) >> 1) & 1);
          tc_fence_after();
          for (int c = 0; c < C::NCH && ok; ++c) {
            const uint32_t slot = (ai0 + c) % C::NA;
            mma_chunk<E, C>(dt, smem_u32(sA + slot * C::SLOT), yop, c, first);
            mma_commit(&b.emptyA[slot]);
          }
          ai = ai0 + C::NCH;
        } else if (ok && fwd) {
          pslot = pi % C::NP;
          ok = mbar_wait(&b.fullP[pslot], (pi / C::NP) & 1);
          tc_fence_after();
          if (ok) ok = mma_block<E, C>(sA, b, ai, dt, smem_u32(sP + pslot * C::PT), first);
          if (ok && t > 0) {
            ok = mbar_wait(&b.yrdy[(t - 1) & 1], ((t - 1) >> 1) & 1);
            tc_fence_after();
            if (ok) ok = mma_block<E, C>(sA, b, ai, dt, yop, first);
          }
        } else if (ok) {
          ok = mbar_wait(&b.yrdy[(t - 1) & 1], ((t - 1) >> 1) & 1);
          tc_fence_after();
          if (ok) ok = mma_block<E, C>(sA, b, ai, dt, yop, first);
        }
        if (ok) {
          mma_commit(&b.mdone[bsel]);
          if (fwd) {
            mma_commit(&b.emptyP[pslot]);
            ++pi;
          }
        }
      }
      if (!ok) atomicExch(status, 2);
      // every issued MMA has completed before TMEM is released
      mma_commit(&b.extra[1]);
      mbar_wait(&b.extra[1], 0);
    }
  } else if constexpr (C::SW) {
    // epilogue, swapped roles: thread <-> tile column n (TMEM lane), group g
    // drains block rows [g*MH, (g+1)*MH) of it
    constexpr int ET_THREADS = 128 * C::EG;
    const int n = 32 * (warp & 3) + lane;
    const int m0 = ((warp - 2) / 4) * C::MH;
    const bool leader = (warp == 2 && lane == 0);
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    uint32_t pe = (uint32_t)nrow;
    bool ok = true;
    for (int t = 0; t < T; ++t) {
      const bool fwd = t < nrow;
      const int o = fwd ? t : nrow - 2 - (t - nrow);
      const int i = a + o;
      const int bsel = t & 1;
      if (ok) ok = mbar_wait(&b.mdone[bsel], (t >> 1) & 1);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      tc_fence_after();
      float v[C::MH];
      if (ok) {
        tmem_cols<C::MH>(tmem + lane_base + bsel * C::ACC + m0, v);
      } else {
#pragma unroll
        for (int q = 0; q < C::MH; ++q) v[q] = 0.f;
      }
      tc_fence_before();
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&b.afree[bsel]);
      if (!fwd) {
        const uint32_t ps = pe % C::NP;
        if (ok) ok = mbar_wait(&b.fullP[ps], (pe / C::NP) & 1);
        ok = __all_sync(0xffffffffu, ok);
        if (ok) row_add<E, C>(sP + ps * C::PT, n, m0, v);  // + y_i
        named_bar_sync(1, ET_THREADS);
        if (ok && leader) mbar_arrive(&b.emptyP[ps]);
        ++pe;
      }
      // one y buffer: the previous row's store must have read it (its MMA
      // finished before mdone of this row)
      if (leader) tma_store_wait_read<0>();
      named_bar_sync(1, ET_THREADS);
      if (ok) row_put<E, C>(sY, n, m0, v);
      fence_proxy_async_smem();
      named_bar_sync(1, ET_THREADS);
      if (leader && ok) {
        mbar_arrive(&b.yrdy[bsel]);
        for (int p = 0; p < C::SP; ++p)
          for (int c = 0; c < C::NCH; ++c)
            tma_store_2d(&tm_w, c * C::CE, p * pplane + i * Kp + n0, sY + p * C::TILE + c * C::TCH);
        tma_store_commit();
        if (t == nrow - 1) {
          tma_store_wait<0>();
          fence_proxy_async_all();
          mbar_arrive(&b.extra[0]);
        }
      }
    }
    if (leader) tma_store_wait<0>();
    if (!ok && leader) atomicExch(status, 3);
  } else {
    // epilogue: EG groups of 4 warps; thread <-> accumulator row, group g
    // drains columns [g*NH, (g+1)*NH)
    constexpr int ET_THREADS = 128 * C::EG;
    int row;
    bool has;
    epi_row<C>(warp, lane, &row, &has);
    const int cb = ((warp - 2) / 4) * C::NH;
    const bool leader = (warp == 2 && lane == 0);
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    uint32_t pe = (uint32_t)nrow;  // P tiles consumed here start after the forward ones
    bool ok = true;
    for (int t = 0; t < T; ++t) {
      const bool fwd = t < nrow;
      const int o = fwd ? t : nrow - 2 - (t - nrow);
      const int i = a + o;
      const int bsel = t & 1;
      if (ok) ok = mbar_wait(&b.mdone[bsel], (t >> 1) & 1);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      tc_fence_after();
      float v[C::NH];
      if (ok) {
        tmem_cols<C::NH>(tmem + lane_base + bsel * C::NT + cb, v);
      } else {
#pragma unroll
        for (int n = 0; n < C::NH; ++n) v[n] = 0.f;
      }
      tc_fence_before();
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&b.afree[bsel]);
      if (!fwd) {
        const uint32_t ps = pe % C::NP;
        if (ok) ok = mbar_wait(&b.fullP[ps], (pe / C::NP) & 1);
        ok = __all_sync(0xffffffffu, ok);
        if (ok && has) {
          const uint8_t* tile = sP + ps * C::PT;
#pragma unroll
          for (int n = 0; n < C::NH; ++n) v[n] += tile_get<E, C>(tile, cb + n, row);
        }
        named_bar_sync(1, ET_THREADS);
        if (ok && leader) mbar_arrive(&b.emptyP[ps]);
        ++pe;
      }
      if (leader) tma_store_wait_read<1>();
      named_bar_sync(1, ET_THREADS);
      uint8_t* ybuf = sY + bsel * C::PT;
      if (ok && has) {
#pragma unroll
        for (int n = 0; n < C::NH; ++n) tile_put<E, C>(ybuf, cb + n, row, v[n]);
      }
      fence_proxy_async_smem();
      named_bar_sync(1, ET_THREADS);
      if (leader && ok) {
        mbar_arrive(&b.yrdy[bsel]);
        for (int p = 0; p < C::SP; ++p)
          for (int c = 0; c < C::NCH; ++c)
            tma_store_2d(&tm_w, c * C::CE, p * pplane + i * Kp + n0, ybuf + p * C::TILE + c * C::TCH);
        tma_store_commit();
        if (t == nrow - 1) {
          tma_store_wait<0>();
          fence_proxy_async_all();
          mbar_arrive(&b.extra[0]);
        }
      }
    }
    if (leader) tma_store_wait<0>();
    if (!ok && leader) atomicExch(status, 3);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, C::TMEM_COLS);
}

// ======================================================================
// Correction kernel, eq. superposition (step 2.3), interior rows:
//   d_i = W_i + U_i X~_s + V_i X~_{s+1}
// written as FP32 into the block-transposed correction panel D by TMA stores
// (no FP64 work on this kernel's critical path); chunk 0 of every segment
// also writes d_{k_s} = X~_s.  The FP64 solution is updated afterwards by
// k_x_update_warp (X (+)= d), a streaming kernel bound by HBM.
// ======================================================================
template <typename E, class C>
__global__ void __launch_bounds__(C::THREADS, 1)
    k_tc_correct(const __grid_constant__ CUtensorMap tm_fac, const __grid_constant__ CUtensorMap tm_w,
                 const __grid_constant__ CUtensorMap tm_d, const E* __restrict__ wp, float* __restrict__ dp, int N,
                 int L, int S, int Kp, int rows_per_cta, const int* done, int* status) {
  if (flag_set(done)) return;
  using CF = Cfg<float, C::M, C::NT, 1, 1>;      // layout of one FP32 d tile
  constexpr int DT = CF::TILE;                    // bytes of one d tile
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  // swapped roles: no staging of W or d in shared memory (the epilogue reads
  // and writes whole rows of them in 16-byte vectors)
  constexpr int NPS = C::SW ? 0 : C::NP;
  constexpr int NDS = C::SW ? 0 : 2;
  uint8_t* sA = sm;
  uint8_t* sP = sA + C::NA * C::SLOT;
  uint8_t* sB = sP + NPS * C::PT;  // X~_s, X~_{s+1} (all planes each)
  uint8_t* sD = sB + 2 * C::PT;    // two FP32 d tiles
  uint64_t* barmem = reinterpret_cast<uint64_t*>(sD + NDS * DT);
  const Bars b = carve<C>(barmem);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(barmem + kBars(C::NA, C::NP));

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n0 = blockIdx.x * C::NT;
  const int s = blockIdx.y;
  const bool has_next = s + 1 < S;
  const int r0 = s * L + 1 + blockIdx.z * rows_per_cta;
  const int r1 = min(r0 + rows_per_cta, s * L + L);
  const int T = max(0, r1 - r0);
  const bool do_iface = blockIdx.z == 0;
  const int fplane = 5 * N * C::M;
  const int pplane = N * Kp;

  if (threadIdx.x == 0) init_bars<C>(b);
  if (warp == 1) {
    tmem_alloc(tslot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tm_fac);
      prefetch_tmap(&tm_w);
      prefetch_tmap(&tm_d);
      bool ok = true;
      // X~_s and X~_{s+1}: the two B operands, loaded once
      mbar_arrive_expect_tx(&b.extra[0], (has_next ? 2 : 1) * C::PT);
      for (int q = 0; q < (has_next ? 2 : 1); ++q)
        for (int p = 0; p < C::SP; ++p)
          for (int c = 0; c < C::NCH; ++c)
            tma_load_2d(sB + q * C::PT + p * C::TILE + c * C::TCH, &tm_w, c * C::CE,
                        p * pplane + ((s + q) * L) * Kp + n0, &b.extra[0]);
      uint32_t ai = 0, pi = 0;
      for (int t = 0; t < T && ok; ++t) {
        const int i = r0 + t;
        if constexpr (!C::SW) ok = load_tile<C>(sP, b, pi, &tm_w, i * Kp + n0, pplane);
        for (int c = 0; c < C::NCH && ok; ++c)
          ok = load_slice<C>(sA, b, ai, &tm_fac, c * C::CE, (FT_U * N + i) * C::M, fplane);
        if (has_next)
          for (int c = 0; c < C::NCH && ok; ++c)
            ok = load_slice<C>(sA, b, ai, &tm_fac, c * C::CE, (FT_V * N + i) * C::M, fplane);
      }
      if (!ok) atomicExch(status, 4);
      mbar_wait(&b.extra[0], 0);
      for (uint32_t q = 0; q < C::NA && q < ai; ++q) {
        const uint32_t last = (ai - 1 - q);
        mbar_wait(&b.fullA[last % C::NA], (last / C::NA) & 1);
      }
      for (uint32_t q = 0; q < C::NP && q < pi; ++q) {
        const uint32_t last = pi - 1 - q;
        mbar_wait(&b.fullP[last % C::NP], (last / C::NP) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = mbar_wait(&b.extra[0], 0);
      tc_fence_after();
      uint32_t ai = 0;
      for (int t = 0; t < T && ok; ++t) {
        const int bsel = t & 1;
        const uint32_t dt = tmem + bsel * C::ACC;
        if (t >= 2) ok = mbar_wait(&b.afree[bsel], ((t >> 1) - 1) & 1);
        tc_fence_after();
        bool first = true;
        if (ok) ok = mma_block<E, C>(sA, b, ai, dt, smem_u32(sB), first);
        if (ok && has_next) ok = mma_block<E, C>(sA, b, ai, dt, smem_u32(sB + C::PT), first);
        if (ok) mma_commit(&b.mdone[bsel]);
      }
      if (!ok) atomicExch(status, 5);
      mma_commit(&b.extra[1]);
      mbar_wait(&b.extra[1], 0);
    }
  } else if constexpr (C::SW) {
    // swapped roles: thread <-> tile column n; W_i read and d_i written as
    // whole row shares straight from / to global memory (an FP64 update of X
    // here, with the 8 epilogue warps of a CTA, measured 2.7x slower than the
    // separate streaming update)
    constexpr int per16 = 16 / C::eb;
    constexpr int NU = C::MH / per16;  // 16-byte units of one plane of a row share
    const int nl = 32 * (warp & 3) + lane;
    const int m0 = ((warp - 2) / 4) * C::MH;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const size_t wplane = (size_t)N * Kp * C::M;
    bool ok = mbar_wait(&b.extra[0], 0);
    ok = __all_sync(0xffffffffu, ok);
    auto put_d = [&](const float (&v)[C::MH], int irow) {
      float4* o = reinterpret_cast<float4*>(dp + ((size_t)irow * Kp + n0 + nl) * C::M + m0);
#pragma unroll
      for (int q = 0; q < C::MH / 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    };
    if (do_iface && ok) {
      float v[C::MH];
#pragma unroll
      for (int q = 0; q < C::MH; ++q) v[q] = 0.f;
      row_add<E, C>(sB, nl, m0, v);  // d_{k_s} = X~_s
      put_d(v, s * L);
    }
    for (int t = 0; t < T; ++t) {
      const int i = r0 + t;
      const int bsel = t & 1;
      // W_i row share, fetched before the wait so its latency overlaps the MMAs
      uint4 whi[NU], wlo[NU];
      const uint4* wsrc = reinterpret_cast<const uint4*>(wp + ((size_t)i * Kp + n0 + nl) * C::M + m0);
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        whi[u] = __ldg(wsrc + u);
        wlo[u] = C::SP == 2 ? __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const E*>(wsrc) + wplane) + u)
                            : make_uint4(0, 0, 0, 0);
      }
      if (ok) ok = mbar_wait(&b.mdone[bsel], (t >> 1) & 1);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      tc_fence_after();
      float v[C::MH];
      if (ok) {
        tmem_cols<C::MH>(tmem + lane_base + bsel * C::ACC + m0, v);
      } else {
#pragma unroll
        for (int q = 0; q < C::MH; ++q) v[q] = 0.f;
      }
      tc_fence_before();
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&b.afree[bsel]);
#pragma unroll
      for (int u = 0; u < NU; ++u) unpack16_add<E, C::SP>(whi[u], wlo[u], &v[u * per16]);
      if (ok) put_d(v, i);
    }
    if (!ok && threadIdx.x == 64) atomicExch(status, 6);
  } else {
    constexpr int ET_THREADS = 128 * C::EG;
    int row;
    bool has;
    epi_row<C>(warp, lane, &row, &has);
    const int cb = ((warp - 2) / 4) * C::NH;
    const bool leader = (warp == 2 && lane == 0);
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    bool ok = mbar_wait(&b.extra[0], 0);
    ok = __all_sync(0xffffffffu, ok);
    int dsel = 0;  // d staging buffer of the next store
    // FP32 values v[] of this thread's row and column share -> staging buffer -> TMA store into D row `irow`
    auto emit = [&](const float (&v)[C::NH], int irow) {
      if (leader) tma_store_wait_read<1>();
      named_bar_sync(1, ET_THREADS);
      uint8_t* dt = sD + dsel * DT;
      if (ok && has) {
#pragma unroll
        for (int n = 0; n < C::NH; ++n) *reinterpret_cast<float*>(dt + kmaj_off<CF>(cb + n, row)) = v[n];
      }
      fence_proxy_async_smem();
      named_bar_sync(1, ET_THREADS);
      if (leader && ok) {
        for (int c = 0; c < CF::NCH; ++c) tma_store_2d(&tm_d, c * CF::CE, irow * Kp + n0, dt + c * CF::TCH);
        tma_store_commit();
      }
      dsel ^= 1;
    };
    if (do_iface) {
      float v[C::NH];
#pragma unroll
      for (int n = 0; n < C::NH; ++n) v[n] = (ok && has) ? tile_get<E, C>(sB, cb + n, row) : 0.f;
      emit(v, s * L);
    }
    uint32_t pe = 0;
    for (int t = 0; t < T; ++t) {
      const int i = r0 + t;
      const int bsel = t & 1;
      if (ok) ok = mbar_wait(&b.mdone[bsel], (t >> 1) & 1);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      tc_fence_after();
      float v[C::NH];
      if (ok) {
        tmem_cols<C::NH>(tmem + lane_base + bsel * C::NT + cb, v);
      } else {
#pragma unroll
        for (int n = 0; n < C::NH; ++n) v[n] = 0.f;
      }
      tc_fence_before();
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&b.afree[bsel]);
      const uint32_t ps = pe % C::NP;
      if (ok) ok = mbar_wait(&b.fullP[ps], (pe / C::NP) & 1);
      ok = __all_sync(0xffffffffu, ok);
      if (ok && has) {
        const uint8_t* tile = sP + ps * C::PT;
#pragma unroll
        for (int n = 0; n < C::NH; ++n) v[n] += tile_get<E, C>(tile, cb + n, row);
      }
      named_bar_sync(1, ET_THREADS);
      if (ok && leader) mbar_arrive(&b.emptyP[ps]);
      ++pe;
      emit(v, i);
    }
    if (leader) tma_store_wait<0>();
    if (!ok && leader) atomicExch(status, 6);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, C::TMEM_COLS);
}

// ======================================================================
// Step 2.2 on the tensor cores (swapped roles): one job per CTA row of the
// grid, one 128-column tile per CTA column.  A job computes
//   v = sum_p  T_p B_p  (+ r panel row)  (+ sum of series terms)
// with up to two products of a work-panel tile T_p (A operand) and an
// interface block B_p (B operand), and writes v to a work-panel row and/or
// an FP32 series-term row.  The three uses, in launch order:
//   F~_s = r_{k_s} + A_{k_s} W_{k_s - 1} + B_{k_s} W_{k_s + 1}  -> panel row k_s (eq. red1)
//   c[l][s] = R[l][s] F~_s                                      -> series terms
//   X~_m = sum_{j in node} c[l][j] + HL_m X~_{l-1} + HR_m X~_{r+1} -> panel row k_m
// (one launch per tree level, Algorithm 1; the node sums of the series terms
// come from k_node_sums, one tile per node).  Series terms are FP32, laid out
// [depth * S][Kp][M] so one thread reads and writes a contiguous row share.
// ======================================================================
struct IfJob {
  int32_t a[2];      // block rows of the A operands (-1: absent)
  int32_t a_src[2];  // 0: a[p] is a work-panel row, 1: a residual-panel row
  int32_t b[2];      // interface block index paired with a[p]
  int32_t add_r;     // r-panel block row added to the result (-1: none)
  int32_t sum_lev;   // series terms c[sum_lev][sum_lo..sum_hi] added (sum_lo > sum_hi: none)
  int32_t sum_lo, sum_hi;
  int32_t out_w;     // work-panel block row receiving the result (-1: none)
  int32_t out_c;     // series-term slot (level * S + s) receiving the result (-1: none)
};

template <typename E, class C>
__global__ void __launch_bounds__(C::THREADS, 1)
    k_tc_ifgemm(const __grid_constant__ CUtensorMap tm_if, const __grid_constant__ CUtensorMap tm_w,
                const __grid_constant__ CUtensorMap tm_r, const IfJob* __restrict__ jobs, int job0, const E* __restrict__ rp, E* __restrict__ wp,
                float* __restrict__ cp, const float* __restrict__ sumbase, int N, int S, int nblk, int Kp,
                const int* done, int* status) {
  static_assert(C::SW, "swapped roles only");
  if (flag_set(done)) return;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = sm;                    // interface-block slices (B operands)
  uint8_t* sT = sA + C::NA * C::SLOT;  // up to two panel tiles (A operands)
  uint64_t* barmem = reinterpret_cast<uint64_t*>(sT + 2 * C::PT);
  const Bars b = carve<C>(barmem);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(barmem + kBars(C::NA, C::NP));

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n0 = blockIdx.x * C::NT;
  const IfJob jb = jobs[job0 + blockIdx.y];
  const int np = (jb.a[0] >= 0 ? 1 : 0) + (jb.a[1] >= 0 ? 1 : 0);
  const int pplane = N * Kp;
  if (threadIdx.x == 0) init_bars<C>(b);
  if (warp == 1) {
    tmem_alloc(tslot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0 && np > 0) {
      prefetch_tmap(&tm_if);
      prefetch_tmap(&tm_w);
      mbar_arrive_expect_tx(&b.extra[0], np * C::PT);
      int k = 0;
      for (int p = 0; p < 2; ++p) {
        if (jb.a[p] < 0) continue;
        const CUtensorMap* tm = jb.a_src[p] ? &tm_r : &tm_w;
        for (int pl = 0; pl < C::SP; ++pl)
          for (int c = 0; c < C::NCH; ++c)
            tma_load_2d(sT + k * C::PT + pl * C::TILE + c * C::TCH, tm, c * C::CE,
                        pl * pplane + jb.a[p] * Kp + n0, &b.extra[0]);
        ++k;
      }
      uint32_t ai = 0;
      bool ok = true;
      for (int p = 0; p < 2 && ok; ++p) {
        if (jb.a[p] < 0) continue;
        for (int c = 0; c < C::NCH && ok; ++c)
          ok = load_slice<C>(sA, b, ai, &tm_if, c * C::CE, jb.b[p] * C::M, nblk * C::M);
      }
      if (!ok) atomicExch(status, 7);
      mbar_wait(&b.extra[0], 0);
      for (uint32_t q = 0; q < C::NA && q < ai; ++q) {
        const uint32_t last = ai - 1 - q;
        mbar_wait(&b.fullA[last % C::NA], (last / C::NA) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && np > 0) {
      bool ok = mbar_wait(&b.extra[0], 0);
      tc_fence_after();
      uint32_t ai = 0;
      bool first = true;
      for (int k = 0; k < np && ok; ++k) ok = mma_block<E, C>(sA, b, ai, tmem, smem_u32(sT + k * C::PT), first);
      if (ok) mma_commit(&b.mdone[0]);
      if (!ok) atomicExch(status, 8);
      mma_commit(&b.extra[1]);
      mbar_wait(&b.extra[1], 0);
    }
  } else {
    constexpr int per16 = 16 / C::eb;
    constexpr int NU = C::MH / per16;
    const int nl = 32 * (warp & 3) + lane;
    const int m0 = ((warp - 2) / 4) * C::MH;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const size_t wplane = (size_t)N * Kp * C::M;
    float v[C::MH];
#pragma unroll
    for (int q = 0; q < C::MH; ++q) v[q] = 0.f;
    bool ok = true;
    if (np > 0) {
      ok = mbar_wait(&b.mdone[0], 0);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      tc_fence_after();
      if (ok) tmem_cols<C::MH>(tmem + lane_base + m0, v);
      tc_fence_before();
    }
    if (jb.add_r >= 0) {
      const uint4* src = reinterpret_cast<const uint4*>(rp + ((size_t)jb.add_r * Kp + n0 + nl) * C::M + m0);
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        const uint4 hi = __ldg(src + u);
        const uint4 lo = C::SP == 2 ? __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const E*>(src) + wplane) + u)
                                    : make_uint4(0, 0, 0, 0);
        unpack16_add<E, C::SP>(hi, lo, &v[u * per16]);
      }
    }
    for (int j = jb.sum_lo; j <= jb.sum_hi; ++j) {
      const float4* src =
          reinterpret_cast<const float4*>(sumbase + (((size_t)jb.sum_lev * S + j) * Kp + n0 + nl) * C::M + m0);
#pragma unroll
      for (int q = 0; q < C::MH / 4; ++q) {
        const float4 t = __ldg(src + q);
        v[4 * q] += t.x;
        v[4 * q + 1] += t.y;
        v[4 * q + 2] += t.z;
        v[4 * q + 3] += t.w;
      }
    }
    if (ok && jb.out_w >= 0) {
      uint4* dst = reinterpret_cast<uint4*>(wp + ((size_t)jb.out_w * Kp + n0 + nl) * C::M + m0);
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        uint4 hi, lo;
        pack16<E, C::SP>(&v[u * per16], hi, lo);
        dst[u] = hi;
        if (C::SP == 2) reinterpret_cast<uint4*>(reinterpret_cast<E*>(dst) + wplane)[u] = lo;
      }
    }
    if (ok && jb.out_c >= 0) {
      float4* dst = reinterpret_cast<float4*>(cp + ((size_t)jb.out_c * Kp + n0 + nl) * C::M + m0);
#pragma unroll
      for (int q = 0; q < C::MH / 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    if (!ok && threadIdx.x == 64) atomicExch(status, 9);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, C::TMEM_COLS);
}

// ======================================================================
// Correction with the interface tiles in tensor memory (split BF16, swapped
// roles, M = 128): X~_s and X~_{s+1} are the A operands of every row's MMAs,
// so the epilogue warps load them once from the work panel and store them
// into TMEM (lane n = tile column n, two block rows per 32-bit column, one
// region per plane); shared memory holds the factor-slice ring and, with WR,
// a ring of W tiles.  TMEM: two accumulators [0, 2M) and four A regions of
// M/2 columns each [2M, 4M).
// ======================================================================
// WR: W_i rows come through a C::NP-stage TMA tile ring (else each epilogue
// thread loads its row share from global memory).
template <class C, bool WR>
__global__ void __launch_bounds__(C::THREADS, 1)
    k_tc_correct_ta(const __grid_constant__ CUtensorMap tm_fac, const __grid_constant__ CUtensorMap tm_w,
                    const __nv_bfloat16* __restrict__ wp, float* __restrict__ dp, double* __restrict__ Xo,
                    float* __restrict__ Drow, int K, int N, int L, int S, int Kp, int rows_per_cta, const int* done,
                    int* status) {
  using E = __nv_bfloat16;
  static_assert(C::SW && C::SP == 2 && C::M == 128 && C::MH == 64, "split BF16, M = 128, swapped roles");
  constexpr int TCOLS = 4 * C::M;
  if (flag_set(done)) return;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = sm;
  uint8_t* sP = sA + C::NA * C::SLOT;
  uint64_t* barmem = reinterpret_cast<uint64_t*>(sP + (WR ? C::NP * C::PT : 0));
  const Bars b = carve<C>(barmem);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(barmem + kBars(C::NA, C::NP));

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n0 = blockIdx.x * C::NT;
  const int s = blockIdx.y;
  const bool has_next = s + 1 < S;
  const int r0 = s * L + 1 + blockIdx.z * rows_per_cta;
  const int r1 = min(r0 + rows_per_cta, s * L + L);
  const int T = max(0, r1 - r0);
  const bool do_iface = blockIdx.z == 0;
  const int fplane = 5 * N * C::M;
  auto acol = [](int q, int pl) { return (uint32_t)(2 * C::M + (2 * q + pl) * (C::M / 2)); };
  if (threadIdx.x == 0) {
    init_bars<C>(b);
    mbar_init(&b.yrdy[0], 4 * C::EG);  // A operands stored by every epilogue warp
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, TCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tm_fac);
      if (WR) prefetch_tmap(&tm_w);
      uint32_t ai = 0, pi = 0;
      bool ok = true;
      const int pplane = N * Kp;
      for (int t = 0; t < T && ok; ++t) {
        const int i = r0 + t;
        if (WR) ok = load_tile<C>(sP, b, pi, &tm_w, i * Kp + n0, pplane);
        for (int c = 0; c < C::NCH && ok; ++c)
          ok = load_slice<C>(sA, b, ai, &tm_fac, c * C::CE, (FT_U * N + i) * C::M, fplane);
        if (has_next)
          for (int c = 0; c < C::NCH && ok; ++c)
            ok = load_slice<C>(sA, b, ai, &tm_fac, c * C::CE, (FT_V * N + i) * C::M, fplane);
      }
      if (!ok) atomicExch(status, 4);
      for (uint32_t q = 0; q < C::NA && q < ai; ++q) {
        const uint32_t last = ai - 1 - q;
        mbar_wait(&b.fullA[last % C::NA], (last / C::NA) & 1);
      }
      for (uint32_t q = 0; q < C::NP && q < pi; ++q) {
        const uint32_t last = pi - 1 - q;
        mbar_wait(&b.fullP[last % C::NP], (last / C::NP) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = mbar_wait(&b.yrdy[0], 0);
      tc_fence_after();
      uint32_t ai = 0;
      for (int t = 0; t < T && ok; ++t) {
        const int bsel = t & 1;
        const uint32_t dt = tmem + bsel * C::ACC;
        if (t >= 2) ok = mbar_wait(&b.afree[bsel], ((t >> 1) - 1) & 1);
        tc_fence_after();
        bool first = true;
        for (int q = 0; q < (has_next ? 2 : 1) && ok; ++q) {
          for (int c = 0; c < C::NCH && ok; ++c) {
            const uint32_t slot = ai % C::NA, use = ai / C::NA;
            ok = mbar_wait(&b.fullA[slot], use & 1);
            if (!ok) break;
            tc_fence_after();
            const uint32_t fb = smem_u32(sA + slot * C::SLOT);
#pragma unroll
            for (int kq = 0; kq < C::CE / C::KS; ++kq) {
              const uint32_t kc = (uint32_t)(c * (C::CE / C::KS) + kq) * (C::KS / 2);  // 2 elements per column
              const uint32_t ahi = tmem + acol(q, 0) + kc, alo = tmem + acol(q, 1) + kc;
              const uint64_t bhi = smem_desc(fb + kq * 32, 16, 1024);
              const uint64_t blo = smem_desc(fb + C::SLICE + kq * 32, 16, 1024);
              mma_f16_ta(dt, ahi, bhi, C::IDESC, first ? 0u : 1u);
              first = false;
              mma_f16_ta(dt, alo, bhi, C::IDESC, 1u);
              mma_f16_ta(dt, ahi, blo, C::IDESC, 1u);
            }
            mma_commit(&b.emptyA[slot]);
            ++ai;
          }
        }
        if (ok) mma_commit(&b.mdone[bsel]);
      }
      if (!ok) atomicExch(status, 5);
      mma_commit(&b.extra[1]);
      mbar_wait(&b.extra[1], 0);
    }
  } else {
    constexpr int per16 = 8;           // bf16 per 16 bytes
    constexpr int NU = C::MH / per16;  // 16-byte units of one plane of a row share
    const int nl = 32 * (warp & 3) + lane;
    const int g = (warp - 2) / 4;
    const int m0 = g * C::MH;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const size_t wplane = (size_t)N * Kp * C::M;
    // Xo != nullptr (the first solve): the result is the solution itself,
    // written as FP64 rows of the row-major X (exact widening; for each block
    // row m the warp's 32 columns are 256 contiguous bytes) instead of the
    // FP32 correction panel; Drow != nullptr: FP32 rows of a row-major
    // [N][M][K] panel (128 contiguous bytes per warp and row m)
    auto store_row = [&](const float (&v)[C::MH], int irow) {
      if (Drow != nullptr) {
        const int n = n0 + nl;
        if (n < K) {
          float* x = Drow + ((size_t)irow * C::M + m0) * K + n;
#pragma unroll
          for (int q0 = 0; q0 < C::MH; q0 += 16) {
#pragma unroll
            for (int q = q0; q < q0 + 16; ++q) x[(size_t)q * K] = v[q];
            asm volatile("" ::: "memory");  // one batch of stores at a time
          }
        }
      } else if (Xo != nullptr) {
        const int n = n0 + nl;
        if (n < K) {
          double* x = Xo + ((size_t)irow * C::M + m0) * K + n;
#pragma unroll
          for (int q0 = 0; q0 < C::MH; q0 += 16) {
#pragma unroll
            for (int q = q0; q < q0 + 16; ++q) x[(size_t)q * K] = f32_to_f64(v[q]);
            asm volatile("" ::: "memory");  // one batch of stores at a time
          }
        }
      } else {
        float4* o = reinterpret_cast<float4*>(dp + ((size_t)irow * Kp + n0 + nl) * C::M + m0);
#pragma unroll
        for (int q = 0; q < C::MH / 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
    };
    // the A operands: rows s*L and (s+1)*L of the work panel into TMEM
    for (int q = 0; q < 2; ++q) {
      if (q == 1 && !has_next) break;
      const uint4* src = reinterpret_cast<const uint4*>(wp + ((size_t)(s + q) * L * Kp + n0 + nl) * C::M + m0);
      uint32_t hi[32], lo[32];
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        const uint4 h4 = __ldg(src + u);
        const uint4 l4 = __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const E*>(src) + wplane) + u);
        hi[4 * u] = h4.x; hi[4 * u + 1] = h4.y; hi[4 * u + 2] = h4.z; hi[4 * u + 3] = h4.w;
        lo[4 * u] = l4.x; lo[4 * u + 1] = l4.y; lo[4 * u + 2] = l4.z; lo[4 * u + 3] = l4.w;
      }
      tmem_st32(tmem + lane_base + acol(q, 0) + g * (C::MH / 2), hi);
      tmem_st32(tmem + lane_base + acol(q, 1) + g * (C::MH / 2), lo);
      if (q == 0 && do_iface) {  // d_{k_s} = X~_s
        float v[C::MH];
#pragma unroll
        for (int e = 0; e < C::MH; ++e) v[e] = 0.f;
#pragma unroll
        for (int u = 0; u < NU; ++u)
          unpack16_add<E, 2>(make_uint4(hi[4 * u], hi[4 * u + 1], hi[4 * u + 2], hi[4 * u + 3]),
                             make_uint4(lo[4 * u], lo[4 * u + 1], lo[4 * u + 2], lo[4 * u + 3]), &v[u * per16]);
        store_row(v, s * L);
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&b.yrdy[0]);
    bool ok = true;
    uint32_t pe = 0;
    for (int t = 0; t < T; ++t) {
      const int i = r0 + t;
      const int bsel = t & 1;
      uint4 whi[WR ? 1 : NU], wlo[WR ? 1 : NU];
      if constexpr (!WR) {
        const uint4* wsrc = reinterpret_cast<const uint4*>(wp + ((size_t)i * Kp + n0 + nl) * C::M + m0);
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          whi[u] = __ldg(wsrc + u);
          wlo[u] = __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const E*>(wsrc) + wplane) + u);
        }
      }
      if (ok) ok = mbar_wait(&b.mdone[bsel], (t >> 1) & 1);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      tc_fence_after();
      float v[C::MH];
      if (ok) {
        tmem_cols<C::MH>(tmem + lane_base + bsel * C::ACC + m0, v);
      } else {
#pragma unroll
        for (int q = 0; q < C::MH; ++q) v[q] = 0.f;
      }
      tc_fence_before();
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&b.afree[bsel]);
      if constexpr (WR) {
        const uint32_t ps = pe % C::NP;
        if (ok) ok = mbar_wait(&b.fullP[ps], (pe / C::NP) & 1);
        ok = __all_sync(0xffffffffu, ok);
        if (ok) row_add<E, C>(sP + ps * C::PT, nl, m0, v);
        named_bar_sync(1, 128 * C::EG);
        if (ok && warp == 2 && lane == 0) mbar_arrive(&b.emptyP[ps]);
        ++pe;
      } else {
#pragma unroll
        for (int u = 0; u < NU; ++u) unpack16_add<E, 2>(whi[u], wlo[u], &v[u * per16]);
      }
      if (ok) store_row(v, i);
    }
    if (!ok && threadIdx.x == 64) atomicExch(status, 6);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, TCOLS);
}

// ======================================================================
// Forward / backward stage 2 for unit stencils (A_i = B_i = I, symmetric P),
// split BF16, swapped roles, M = 128.  The correction of step 2.3 folds into
// a backward pass that forms X directly once the interface values are known:
//   forward  (k_tc_fwd):  y_i = Dinv_i (r_i + y_{i-1})            -> work panel row i
//                         W_a = sum_i Z_i r_i, Z_i = U_i^T        -> residual panel row a
//   step 2.2 (unchanged but F~ reads W_a from the residual panel; W_b = y_b)
//   backward (k_tc_bwd):  X_i = y_i + Y_i X~_s + G_i X_{i+1},  X_{b+1} = X~_{s+1}
// (a..b: a segment's interior rows).  Z_i is block row a of the interior's
// inverse: U_i = [P_II^-1]_{i,a} (A_a = I) and P_II is symmetric.  Y_i =
// E_i Y_{i-1}, Y_a = E_a, is the forward response to the left interface
// value.  In exact arithmetic X equals eq. superposition's W + U X~_s + V
// X~_{s+1}; the panel traffic per solve drops from 24 to 16 bytes per
// unknown (no W panel written and read back, no separate correction pass).
// Factor set [2 planes][4][N][M][M]: Dinv, G, Z, Y (FB_*).
// ======================================================================
enum { FB_DINV = 0, FB_G = 1, FB_Z = 2, FB_Y = 3 };

template <class C>
__global__ void __launch_bounds__(C::THREADS, 1)
    k_tc_fwd(const __grid_constant__ CUtensorMap tm_fac, const __grid_constant__ CUtensorMap tm_r,
             const __grid_constant__ CUtensorMap tm_w, int N, int L, int Kp, const int* done, int* status) {
  using E = __nv_bfloat16;
  static_assert(C::SW && C::SP == 2 && C::M == 128 && C::YB == 1, "split BF16, M = 128, swapped roles");
  constexpr int TCOLS = 4 * C::M;  // two row accumulators, the W_a accumulator (and a spare region)
  if (flag_set(done)) return;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = sm;
  uint8_t* sP = sA + C::NA * C::SLOT;
  uint8_t* sY = sP + C::NP * C::PT;
  uint64_t* barmem = reinterpret_cast<uint64_t*>(sY + C::PT);
  const Bars b = carve<C>(barmem);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(barmem + kBars(C::NA, C::NP));

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n0 = blockIdx.x * C::NT;
  const int s = blockIdx.y;
  const int a = s * L + 1;   // first interior row
  const int nrow = L - 1;    // interior rows (>= 1)
  const int fplane = 4 * N * C::M;
  const int pplane = N * Kp;
  const uint32_t zacc = 2 * C::ACC;  // TMEM columns of the W_a accumulator
  if (threadIdx.x == 0) init_bars<C>(b);
  if (warp == 1) {
    tmem_alloc(tslot, TCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tm_fac);
      prefetch_tmap(&tm_r);
      prefetch_tmap(&tm_w);
      uint32_t ai = 0, pi = 0;
      bool ok = true;
      for (int t = 0; t < nrow && ok; ++t) {
        const int i = a + t;
        ok = load_tile<C>(sP, b, pi, &tm_r, i * Kp + n0, pplane);
        for (int c = 0; c < C::NCH && ok; ++c)
          ok = load_slice<C>(sA, b, ai, &tm_fac, c * C::CE, (FB_DINV * N + i) * C::M, fplane);
        for (int c = 0; c < C::NCH && ok; ++c)
          ok = load_slice<C>(sA, b, ai, &tm_fac, c * C::CE, (FB_Z * N + i) * C::M, fplane);
      }
      if (!ok) atomicExch(status, 11);
      for (uint32_t q = 0; q < C::NA && q < ai; ++q) {
        const uint32_t last = ai - 1 - q;
        mbar_wait(&b.fullA[last % C::NA], (last / C::NA) & 1);
      }
      for (uint32_t q = 0; q < C::NP && q < pi; ++q) {
        const uint32_t last = pi - 1 - q;
        mbar_wait(&b.fullP[last % C::NP], (last / C::NP) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t ai = 0, pi = 0;
      bool ok = true, zfirst = true;
      for (int t = 0; t < nrow && ok; ++t) {
        const int bsel = t & 1;
        const uint32_t dt = tmem + bsel * C::ACC;
        if (t >= 2) ok = mbar_wait(&b.afree[bsel], ((t >> 1) - 1) & 1);
        tc_fence_after();
        const uint32_t pslot = pi % C::NP;
        if (ok) ok = mbar_wait(&b.fullP[pslot], (pi / C::NP) & 1);
        tc_fence_after();
        const uint32_t ptile = smem_u32(sP + pslot * C::PT);
        bool first = true;
        // Dinv_i r_i (+ Dinv_i y_{i-1}): each Dinv slice serves both products
        const uint32_t ai0 = ai;
        for (int c = 0; c < C::NCH && ok; ++c) {
          const uint32_t q = ai0 + c, slot = q % C::NA;
          ok = mbar_wait(&b.fullA[slot], (q / C::NA) & 1);
          tc_fence_after();
          if (ok) mma_chunk<E, C>(dt, smem_u32(sA + slot * C::SLOT), ptile, c, first);
        }
        if (ok && t > 0) {
          ok = mbar_wait(&b.yrdy[(t - 1) & 1], ((t - 1) >> 1) & 1);
          tc_fence_after();
          for (int c = 0; c < C::NCH && ok; ++c)
            mma_chunk<E, C>(dt, smem_u32(sA + ((ai0 + c) % C::NA) * C::SLOT), smem_u32(sY), c, first);
        }
        if (!ok) break;
        for (int c = 0; c < C::NCH; ++c) mma_commit(&b.emptyA[(ai0 + c) % C::NA]);
        mma_commit(&b.mdone[bsel]);
        ai = ai0 + C::NCH;
        // Z_i r_i into the W_a accumulator (off the recurrence's critical path)
        for (int c = 0; c < C::NCH && ok; ++c) {
          const uint32_t slot = ai % C::NA;
          ok = mbar_wait(&b.fullA[slot], (ai / C::NA) & 1);
          tc_fence_after();
          if (ok) {
            mma_chunk<E, C>(tmem + zacc, smem_u32(sA + slot * C::SLOT), ptile, c, zfirst);
            mma_commit(&b.emptyA[slot]);
          }
          ++ai;
        }
        if (ok) {
          mma_commit(&b.emptyP[pslot]);
          ++pi;
        }
      }
      if (ok) mma_commit(&b.extra[0]);  // the W_a accumulator is complete
      if (!ok) atomicExch(status, 12);
      mma_commit(&b.extra[1]);
      mbar_wait(&b.extra[1], 0);
    }
  } else {
    constexpr int ET_THREADS = 128 * C::EG;
    const int n = 32 * (warp & 3) + lane;
    const int m0 = ((warp - 2) / 4) * C::MH;
    const bool leader = (warp == 2 && lane == 0);
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    bool ok = true;
    for (int t = 0; t < nrow; ++t) {
      const int i = a + t;
      const int bsel = t & 1;
      if (ok) ok = mbar_wait(&b.mdone[bsel], (t >> 1) & 1);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      tc_fence_after();
      float v[C::MH];
      if (ok) {
        tmem_cols<C::MH>(tmem + lane_base + bsel * C::ACC + m0, v);
      } else {
#pragma unroll
        for (int q = 0; q < C::MH; ++q) v[q] = 0.f;
      }
      tc_fence_before();
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&b.afree[bsel]);
      // one y buffer: the previous row's store must have read it
      if (leader) tma_store_wait_read<0>();
      named_bar_sync(1, ET_THREADS);
      if (ok) row_put<E, C>(sY, n, m0, v);
      fence_proxy_async_smem();
      named_bar_sync(1, ET_THREADS);
      if (leader && ok) {
        mbar_arrive(&b.yrdy[bsel]);
        for (int p = 0; p < C::SP; ++p)
          for (int c = 0; c < C::NCH; ++c)
            tma_store_2d(&tm_w, c * C::CE, p * pplane + i * Kp + n0, sY + p * C::TILE + c * C::TCH);
        tma_store_commit();
      }
    }
    // W_a = sum_i Z_i r_i -> residual panel row a
    if (ok) ok = mbar_wait(&b.extra[0], 0);
    ok = __all_sync(0xffffffffu, ok);
    tc_fence_after();
    float v[C::MH];
    if (ok) {
      tmem_cols<C::MH>(tmem + lane_base + zacc + m0, v);
    } else {
#pragma unroll
      for (int q = 0; q < C::MH; ++q) v[q] = 0.f;
    }
    tc_fence_before();
    if (leader) tma_store_wait_read<0>();
    named_bar_sync(1, ET_THREADS);
    if (ok) row_put<E, C>(sY, n, m0, v);
    fence_proxy_async_smem();
    named_bar_sync(1, ET_THREADS);
    if (leader && ok) {
      for (int p = 0; p < C::SP; ++p)
        for (int c = 0; c < C::NCH; ++c)
          tma_store_2d(&tm_r, c * C::CE, p * pplane + a * Kp + n0, sY + p * C::TILE + c * C::TCH);
      tma_store_commit();
    }
    if (leader) tma_store_wait<0>();
    if (!ok && leader) atomicExch(status, 13);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, TCOLS);
}

// Backward pass: X_i = y_i + Y_i X~_s + G_i X_{i+1} for i = b..a with
// X_{b+1} = X~_{s+1} (zero for the last segment).  X~_s lives in TMEM as the A
// operand of every Y product; the recurrence operand X_{i+1} is a shared-
// memory tile (X~_{s+1} by TMA for the first row, then each row written by
// the epilogue); y_i comes through the panel ring and is added in the
// epilogue.  Each X_i goes to the row-major FP32 panel Drow ([N][M][K]), the
// interface row k_s takes X~_s.
template <class C>
__global__ void __launch_bounds__(C::THREADS, 1)
    k_tc_bwd(const __grid_constant__ CUtensorMap tm_fac, const __grid_constant__ CUtensorMap tm_w,
             const __nv_bfloat16* __restrict__ wp, float* __restrict__ Drow, int K, int N, int L, int S, int Kp,
             const int* done, int* status) {
  using E = __nv_bfloat16;
  static_assert(C::SW && C::SP == 2 && C::M == 128 && C::MH == 64, "split BF16, M = 128, swapped roles");
  constexpr int TCOLS = 4 * C::M;
  if (flag_set(done)) return;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = sm;
  uint8_t* sP = sA + C::NA * C::SLOT;
  uint8_t* sY = sP + C::NP * C::PT;
  uint64_t* barmem = reinterpret_cast<uint64_t*>(sY + C::PT);
  const Bars b = carve<C>(barmem);
  // beyond the common set: X~_s stored into TMEM by every epilogue warp
  uint64_t* a_rdy = barmem + kBars(C::NA, C::NP);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(barmem + kBars(C::NA, C::NP) + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n0 = blockIdx.x * C::NT;
  const int s = blockIdx.y;
  const bool has_next = s + 1 < S;
  const int a = s * L + 1, nrow = L - 1;
  const int bl = a + nrow - 1;  // last interior row
  const int fplane = 4 * N * C::M;
  const int pplane = N * Kp;
  auto acol = [](int pl) { return (uint32_t)(2 * C::M + pl * (C::M / 2)); };
  if (threadIdx.x == 0) {
    init_bars<C>(b);
    mbar_init(a_rdy, 4 * C::EG);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, TCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tm_fac);
      prefetch_tmap(&tm_w);
      bool ok = true;
      if (has_next) {  // X~_{s+1}: the first recurrence operand
        mbar_arrive_expect_tx(&b.extra[0], C::PT);
        for (int p = 0; p < C::SP; ++p)
          for (int c = 0; c < C::NCH; ++c)
            tma_load_2d(sY + p * C::TILE + c * C::TCH, &tm_w, c * C::CE, p * pplane + (s + 1) * L * Kp + n0,
                        &b.extra[0]);
      }
      uint32_t ai = 0, pi = 0;
      for (int t = 0; t < nrow && ok; ++t) {
        const int i = bl - t;
        ok = load_tile<C>(sP, b, pi, &tm_w, i * Kp + n0, pplane);
        for (int c = 0; c < C::NCH && ok; ++c)
          ok = load_slice<C>(sA, b, ai, &tm_fac, c * C::CE, (FB_Y * N + i) * C::M, fplane);
        if (t > 0 || has_next)
          for (int c = 0; c < C::NCH && ok; ++c)
            ok = load_slice<C>(sA, b, ai, &tm_fac, c * C::CE, (FB_G * N + i) * C::M, fplane);
      }
      if (!ok) atomicExch(status, 14);
      if (has_next) mbar_wait(&b.extra[0], 0);
      for (uint32_t q = 0; q < C::NA && q < ai; ++q) {
        const uint32_t last = ai - 1 - q;
        mbar_wait(&b.fullA[last % C::NA], (last / C::NA) & 1);
      }
      for (uint32_t q = 0; q < C::NP && q < pi; ++q) {
        const uint32_t last = pi - 1 - q;
        mbar_wait(&b.fullP[last % C::NP], (last / C::NP) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = mbar_wait(a_rdy, 0);
      tc_fence_after();
      uint32_t ai = 0;
      for (int t = 0; t < nrow && ok; ++t) {
        const int bsel = t & 1;
        const uint32_t dt = tmem + bsel * C::ACC;
        if (t >= 2) ok = mbar_wait(&b.afree[bsel], ((t >> 1) - 1) & 1);
        tc_fence_after();
        bool first = true;
        // Y_i X~_s: X~_s from TMEM (two BF16 values per 32-bit column)
        for (int c = 0; c < C::NCH && ok; ++c) {
          const uint32_t slot = ai % C::NA;
          ok = mbar_wait(&b.fullA[slot], (ai / C::NA) & 1);
          if (!ok) break;
          tc_fence_after();
          const uint32_t fb = smem_u32(sA + slot * C::SLOT);
#pragma unroll
          for (int kq = 0; kq < C::CE / C::KS; ++kq) {
            const uint32_t kc = (uint32_t)(c * (C::CE / C::KS) + kq) * (C::KS / 2);
            const uint32_t ahi = tmem + acol(0) + kc, alo = tmem + acol(1) + kc;
            const uint64_t bhi = smem_desc(fb + kq * 32, 16, 1024);
            const uint64_t blo = smem_desc(fb + C::SLICE + kq * 32, 16, 1024);
            mma_f16_ta(dt, ahi, bhi, C::IDESC, first ? 0u : 1u);
            first = false;
            mma_f16_ta(dt, alo, bhi, C::IDESC, 1u);
            mma_f16_ta(dt, ahi, blo, C::IDESC, 1u);
          }
          mma_commit(&b.emptyA[slot]);
          ++ai;
        }
        // G_i X_{i+1}: the recurrence operand in shared memory
        if (ok && (t > 0 || has_next)) {
          ok = t == 0 ? mbar_wait(&b.extra[0], 0) : mbar_wait(&b.yrdy[(t - 1) & 1], ((t - 1) >> 1) & 1);
          tc_fence_after();
          if (ok) ok = mma_block<E, C>(sA, b, ai, dt, smem_u32(sY), first);
        }
        if (ok) mma_commit(&b.mdone[bsel]);
      }
      if (!ok) atomicExch(status, 15);
      mma_commit(&b.extra[1]);
      mbar_wait(&b.extra[1], 0);
    }
  } else {
    constexpr int ET_THREADS = 128 * C::EG;
    constexpr int per16 = 8;           // bf16 per 16 bytes
    constexpr int NU = C::MH / per16;  // 16-byte units of one plane of a row share
    const int nl = 32 * (warp & 3) + lane;
    const int g = (warp - 2) / 4;
    const int m0 = g * C::MH;
    const bool leader = (warp == 2 && lane == 0);
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const size_t wplane = (size_t)N * Kp * C::M;
    const int n = n0 + nl;
    auto store_row = [&](const float (&v)[C::MH], int irow) {
      if (n < K) {
        float* x = Drow + ((size_t)irow * C::M + m0) * K + n;
#pragma unroll
        for (int q0 = 0; q0 < C::MH; q0 += 16) {
#pragma unroll
          for (int q = q0; q < q0 + 16; ++q) x[(size_t)q * K] = v[q];
          asm volatile("" ::: "memory");  // one batch of stores at a time
        }
      }
    };
    {  // X~_s into TMEM (the A operand of the Y products); d_{k_s} = X~_s
      const uint4* src = reinterpret_cast<const uint4*>(wp + ((size_t)s * L * Kp + n0 + nl) * C::M + m0);
      uint32_t hi[32], lo[32];
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        const uint4 h4 = __ldg(src + u);
        const uint4 l4 = __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const E*>(src) + wplane) + u);
        hi[4 * u] = h4.x; hi[4 * u + 1] = h4.y; hi[4 * u + 2] = h4.z; hi[4 * u + 3] = h4.w;
        lo[4 * u] = l4.x; lo[4 * u + 1] = l4.y; lo[4 * u + 2] = l4.z; lo[4 * u + 3] = l4.w;
      }
      tmem_st32(tmem + lane_base + acol(0) + g * (C::MH / 2), hi);
      tmem_st32(tmem + lane_base + acol(1) + g * (C::MH / 2), lo);
      float v[C::MH];
#pragma unroll
      for (int e = 0; e < C::MH; ++e) v[e] = 0.f;
#pragma unroll
      for (int u = 0; u < NU; ++u)
        unpack16_add<E, 2>(make_uint4(hi[4 * u], hi[4 * u + 1], hi[4 * u + 2], hi[4 * u + 3]),
                           make_uint4(lo[4 * u], lo[4 * u + 1], lo[4 * u + 2], lo[4 * u + 3]), &v[u * per16]);
      store_row(v, s * L);
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(a_rdy);
    bool ok = true;
    uint32_t pe = 0;
    for (int t = 0; t < nrow; ++t) {
      const int i = bl - t;
      const int bsel = t & 1;
      if (ok) ok = mbar_wait(&b.mdone[bsel], (t >> 1) & 1);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      tc_fence_after();
      float v[C::MH];
      if (ok) {
        tmem_cols<C::MH>(tmem + lane_base + bsel * C::ACC + m0, v);
      } else {
#pragma unroll
        for (int q = 0; q < C::MH; ++q) v[q] = 0.f;
      }
      tc_fence_before();
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&b.afree[bsel]);
      const uint32_t ps = pe % C::NP;
      if (ok) ok = mbar_wait(&b.fullP[ps], (pe / C::NP) & 1);
      ok = __all_sync(0xffffffffu, ok);
      if (ok) row_add<E, C>(sP + ps * C::PT, nl, m0, v);  // + y_i
      // the MMAs of this row (the last readers of sY) have completed: mdone
      named_bar_sync(1, ET_THREADS);
      if (ok && leader) mbar_arrive(&b.emptyP[ps]);
      ++pe;
      if (ok) row_put<E, C>(sY, nl, m0, v);  // X_i: the next row's recurrence operand
      fence_proxy_async_smem();
      named_bar_sync(1, ET_THREADS);
      if (ok && leader) mbar_arrive(&b.yrdy[bsel]);
      if (ok) store_row(v, i);
    }
    if (!ok && leader) atomicExch(status, 16);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, TCOLS);
}

// Split-BF16 copies of Dinv, G, Z = U^T and Y, [2][4][N][M][M].
__global__ void k_cast_fb(const double* __restrict__ D, const double* __restrict__ G, const double* __restrict__ U,
                          const double* __restrict__ Y, __nv_bfloat16* __restrict__ out, size_t nb, int M) {
  const size_t n = 4 * nb, MM = (size_t)M * M;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t w = e / nb, o = e % nb;
    double x;
    if (w == FB_Z) {  // element (m, k) of Z_i is element (k, m) of U_i
      const size_t blk = o / MM, r = o % MM;
      x = U[blk * MM + (r % M) * M + r / M];
    } else {
      x = (w == FB_DINV ? D : w == FB_G ? G : Y)[o];
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn((float)x);
    out[e] = hi;
    out[e + n] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(hi)));
  }
}

// X (+)= d: the block-transposed FP32 correction panel into the caller's
// row-major FP64 solution, one warp per (block row j, 8 rows m, 32 columns n): lane n
// reads its 8 FP32 corrections (32 contiguous bytes of the block-transposed
// panel) and updates rows m0..m0+7 of column n of the row-major solution
// (each a coalesced 256-byte row); no shared memory, no barrier.  The panel
// has Mt >= M rows per block row (Mt % 8 == 0); rows past M are padding.
__global__ void __launch_bounds__(256) k_x_update_warp(const float* __restrict__ d, double* __restrict__ X, int N,
                                                       int M, int Mt, int K, int Kp, int accumulate, const int* done) {
  if (flag_set(done)) return;
  const int lane = threadIdx.x % 32;
  const int tn = (K + 31) / 32, tm = (M + 7) / 8;
  const int64_t nitem = (int64_t)N * tm * tn;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t it = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; it < nitem; it += warps) {
    const int n = (int)(it % tn) * 32 + lane;
    const int m0 = (int)((it / tn) % tm) * 8;
    const int64_t j = it / ((int64_t)tn * tm);
    if (n >= K) continue;
    const float4* src = reinterpret_cast<const float4*>(d + ((size_t)j * Kp + n) * Mt + m0);
    const float4 a = __ldg(src), b = __ldg(src + 1);
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    double* x = X + ((size_t)j * M + m0) * K + n;
    const int rows = min(8, M - m0);
    if (accumulate) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < rows) x[(size_t)q * K] += f32_to_f64(v[q]);
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < rows) x[(size_t)q * K] = f32_to_f64(v[q]);
    }
  }
}

// ======================================================================
// Step 2.2 on the CUDA cores (FP32), block-transposed panels of type E with
// SP planes (plane stride `ps` elements).  Each thread owns a 4 x 8 register
// tile (4 block rows x 8 columns); the FP32 interface blocks are stored
// transposed (element (m, k) at k*M + m) so the four rows of one k are one
// 16-byte load, and the panel tile is read from shared memory as two
// broadcast 16-byte loads per k.
// ======================================================================
template <typename E, int SP>
__device__ __forceinline__ float pget(const E* base, size_t idx, size_t ps) {
  float v = ET<E>::tof(base[idx]);
  if (SP == 2) v += ET<E>::tof(base[idx + ps]);
  return v;
}

// acc[i][j] += sum_k At[k][r0+i] * pan[k][c0+j]
template <int KT>
__device__ __forceinline__ void mt_gemm(float (&acc)[4][8], const float* __restrict__ At, int M, int r0,
                                        const float* pan, int c0) {
#pragma unroll 4
  for (int k = 0; k < M; ++k) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(At + (size_t)k * M + r0));
    const float4 p0 = *reinterpret_cast<const float4*>(pan + k * KT + c0);
    const float4 p1 = *reinterpret_cast<const float4*>(pan + k * KT + c0 + 4);
    const float av[4] = {a.x, a.y, a.z, a.w};
    const float pv[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], pv[j], acc[i][j]);
  }
}

// F~_s = r_K + A_K W_{K-1} + B_K W_{K+1};  c[l][s] = R[l][s] F~_s  (FP32, c row-major [M][Kp])
template <typename E, int SP, int KT>
__global__ void k_tc_iface(const E* __restrict__ r, const E* __restrict__ w, const float* __restrict__ tAK,
                           const float* __restrict__ tBK, const float* __restrict__ tR,
                           const int* __restrict__ mid_level, float* __restrict__ cbuf, int N, int M, int S, int L,
                           int Kp, const int* done) {
  if (flag_set(done)) return;
  extern __shared__ __align__(16) float fsm[];
  constexpr int CGS = KT / 8;
  const int t = threadIdx.x, r0 = (t / CGS) * 4, c0 = (t % CGS) * 8;
  const int s = blockIdx.x, col0 = blockIdx.y * KT;
  const int Kr = s * L;
  const size_t ps = (size_t)N * Kp * M;
  float* pa = fsm;
  float* pb = fsm + M * KT;
  float* pt = fsm + 2 * M * KT;
  const bool hasL = s > 0 && L > 1, hasR = Kr + 1 < N && L > 1;
  for (int e = t; e < M * KT; e += blockDim.x) {
    const int mm = e % M, n = e / M;  // coalesced along m
    const size_t off = (size_t)(col0 + n) * M + mm;
    pa[mm * KT + n] = hasL ? pget<E, SP>(w, (size_t)(Kr - 1) * Kp * M + off, ps) : 0.f;
    pb[mm * KT + n] = hasR ? pget<E, SP>(w, (size_t)(Kr + 1) * Kp * M + off, ps) : 0.f;
    pt[mm * KT + n] = pget<E, SP>(r, (size_t)Kr * Kp * M + off, ps);
  }
  __syncthreads();
  const size_t MM = (size_t)M * M;
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = pt[(r0 + i) * KT + c0 + j];
  if (hasL) mt_gemm<KT>(acc, tAK + s * MM, M, r0, pa, c0);
  if (hasR) mt_gemm<KT>(acc, tBK + s * MM, M, r0, pb, c0);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) pt[(r0 + i) * KT + c0 + j] = acc[i][j];
  __syncthreads();
  const int top = mid_level[s];
  for (int lev = 0; lev <= top; ++lev) {
    float cc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) cc[i][j] = 0.f;
    mt_gemm<KT>(cc, tR + ((size_t)lev * S + s) * MM, M, r0, pt, c0);
    float* out = cbuf + ((size_t)lev * S + s) * M * Kp + (size_t)r0 * Kp + col0 + c0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float4* o = reinterpret_cast<float4*>(out + (size_t)i * Kp);
      o[0] = make_float4(cc[i][0], cc[i][1], cc[i][2], cc[i][3]);
      o[1] = make_float4(cc[i][4], cc[i][5], cc[i][6], cc[i][7]);
    }
  }
}

// X~_m = sum_{j in [l, r]} c[level][j] + HL_m X~_{l-1} + HR_m X~_{r+1}, written
// into the work panel's interface row k_m (all planes).
template <typename E, int SP, int KT>
__global__ void k_tc_dichotomy(E* __restrict__ w, const float* __restrict__ cbuf, const float* __restrict__ tHL,
                               const float* __restrict__ tHR, const int* __restrict__ nodes, int lev, int node_off,
                               int N, int M, int S, int L, int Kp, const int* done) {
  if (flag_set(done)) return;
  extern __shared__ __align__(16) float fsm[];
  constexpr int CGS = KT / 8;
  const int t = threadIdx.x, r0 = (t / CGS) * 4, c0 = (t % CGS) * 8;
  const int q = node_off + blockIdx.x;
  const int l = nodes[3 * q], r = nodes[3 * q + 1], mid = nodes[3 * q + 2];
  const int col0 = blockIdx.y * KT;
  const size_t ps = (size_t)N * Kp * M;
  float* pl = fsm;
  float* pr = fsm + M * KT;
  const bool hl = l > 0, hr = r < S - 1;
  for (int e = t; e < M * KT; e += blockDim.x) {
    const int mm = e % M, n = e / M;
    const size_t off = (size_t)(col0 + n) * M + mm;
    pl[mm * KT + n] = hl ? pget<E, SP>(w, (size_t)(l - 1) * L * Kp * M + off, ps) : 0.f;
    pr[mm * KT + n] = hr ? pget<E, SP>(w, (size_t)(r + 1) * L * Kp * M + off, ps) : 0.f;
  }
  __syncthreads();
  const size_t MM = (size_t)M * M;
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  for (int j = l; j <= r; ++j) {
    const float* cj = cbuf + ((size_t)lev * S + j) * M * Kp + (size_t)r0 * Kp + col0 + c0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 u0 = *reinterpret_cast<const float4*>(cj + (size_t)i * Kp);
      const float4 u1 = *reinterpret_cast<const float4*>(cj + (size_t)i * Kp + 4);
      acc[i][0] += u0.x; acc[i][1] += u0.y; acc[i][2] += u0.z; acc[i][3] += u0.w;
      acc[i][4] += u1.x; acc[i][5] += u1.y; acc[i][6] += u1.z; acc[i][7] += u1.w;
    }
  }
  if (hl) mt_gemm<KT>(acc, tHL + (size_t)mid * MM, M, r0, pl, c0);
  if (hr) mt_gemm<KT>(acc, tHR + (size_t)mid * MM, M, r0, pr, c0);
  // rows r0..r0+3 are contiguous in the block-transposed panel: write them per column
  E* out = w + (size_t)mid * L * Kp * M;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const size_t off = (size_t)(col0 + c0 + j) * M + r0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (SP == 2) {
        E hi, lo;
        ET<E>::split(acc[i][j], hi, lo);
        out[off + i] = hi;
        out[off + i + ps] = lo;
      } else {
        out[off + i] = ET<E>::from(acc[i][j]);
      }
    }
  }
}

// FP32 transposed copies of the interface blocks (element (m, k) at k*M + m).
// Entry e of a block array padded from M x M to Mt x Mt blocks (zero rows and
// columns past M): the padded system holds the real one in its leading rows
// and columns, and every padded unknown stays zero through the solve.
__device__ __forceinline__ double padded(const double* __restrict__ src, size_t e, int M, int Mt) {
  const size_t MMt = (size_t)Mt * Mt;
  const size_t b = e / MMt, o = e % MMt;
  const int r = (int)(o / Mt), c = (int)(o % Mt);
  return (r < M && c < M) ? src[b * M * M + (size_t)r * M + c] : 0.0;
}

// Transposed FP32 copy of nblk blocks, padded to Mt x Mt.
__global__ void k_cast_transpose(const double* __restrict__ src, float* __restrict__ dst, size_t nblk, int M, int Mt) {
  const size_t MMt = (size_t)Mt * Mt, n = nblk * MMt;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t bI = e / MMt, o = e % MMt;
    const int k = (int)(o / Mt), m = (int)(o % Mt);
    dst[e] = (k < M && m < M) ? (float)src[bI * M * M + (size_t)m * M + k] : 0.f;
  }
}

// ======================================================================
// host side
// ======================================================================
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

bt_status make_map(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int eb, uint64_t inner, uint64_t outer,
                   uint32_t box_inner, uint32_t box_outer) {
  auto enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return BT_ERR_CUDA;
  }
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * (uint64_t)eb};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return BT_ERR_CUDA;
  }
  return BT_OK;
}

// [SP][5][N][M][M] rounded factor copies (Dinv, E, G, U, V); plane 1 holds the
// rounding remainder of plane 0.
template <typename E, int SP>
__global__ void k_cast_factors(const double* __restrict__ D, const double* __restrict__ Ee,
                               const double* __restrict__ G, const double* __restrict__ U,
                               const double* __restrict__ V, E* __restrict__ out, size_t nb, int M, int Mt) {
  // nb: entries of one padded factor array (N Mt Mt)
  const size_t n = 5 * nb;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t w = e / nb, o = e % nb;
    const double* src = w == 0 ? D : w == 1 ? Ee : w == 2 ? G : w == 3 ? U : V;
    const double x = padded(src, o, M, Mt);
    if (SP == 2) {
      E hi, lo;
      // remainder taken against the FP64 value, then rounded
      ET<E>::split((float)x, hi, lo);
      const double r = x - (double)ET<E>::tof(hi);
      lo = ET<E>::from((float)r);
      out[e] = hi;
      out[e + n] = lo;
    } else {
      out[e] = ET<E>::from((float)x);
    }
  }
}

// Split-BF16 copy of blocks padded to Mt x Mt (n padded entries): plane 0 at
// dst, plane 1 (remainder) at dst + plane.
__global__ void k_cast_split(const double* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t n, size_t plane,
                             int M, int Mt) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double x = padded(src, e, M, Mt);
    const __nv_bfloat16 hi = __float2bfloat16_rn((float)x);
    dst[e] = hi;
    dst[e + plane] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(hi)));
  }
}

// Sum of the series terms of every tree node, sum_{j = l..r} c[level][j], into
// csum[q] ([Kp][M] FP32 per node q): one CTA per (1024-entry chunk, node).
__global__ void __launch_bounds__(256) k_node_sums(const float* __restrict__ c, float* __restrict__ csum,
                                                   const int* __restrict__ nodes, const int* __restrict__ mid_level,
                                                   int S, size_t tile, const int* done) {
  if (flag_set(done)) return;
  const int q = blockIdx.y;
  const int l = nodes[3 * q], r = nodes[3 * q + 1], lev = mid_level[nodes[3 * q + 2]];
  const size_t e = (size_t)blockIdx.x * 1024 + 4 * threadIdx.x;
  if (e >= tile) return;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const float* src = c + ((size_t)lev * S + l) * tile + e;
#pragma unroll 8
  for (int j = l; j <= r; ++j, src += tile) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(src));
    acc.x += t.x;
    acc.y += t.y;
    acc.z += t.z;
    acc.w += t.w;
  }
  *reinterpret_cast<float4*>(csum + (size_t)q * tile + e) = acc;
}

// Interface blocks for the tensor-core step 2.2 and its job table (once per handle).
bt_status make_tc_interface(bt_handle_s* h, cudaStream_t st) {
  if (h->tc_if_bf16x3) return BT_OK;
  const int S = (int)h->S, L = (int)h->L, N = (int)h->N, depth = h->depth;
  const int Mt = tc_M(h);
  const size_t MM = (size_t)Mt * Mt;
  const size_t nblk = (size_t)(4 + depth) * S;
  void* buf = nullptr;
  BT_TRY(h->arena.alloc(&buf, 2 * nblk * MM * sizeof(__nv_bfloat16)));
  __nv_bfloat16* d = reinterpret_cast<__nv_bfloat16*>(buf);
  const size_t plane = nblk * MM;
  struct Src {
    const double* p;
    size_t nb;
  } srcs[] = {{h->AK, (size_t)S}, {h->BK, (size_t)S}, {h->R, (size_t)depth * S}, {h->HL, (size_t)S}, {h->HR, (size_t)S}};
  size_t at = 0;
  for (const Src& q : srcs) {
    k_cast_split<<<512, 256, 0, st>>>(q.p, d + at * MM, q.nb * MM, plane, (int)h->M, Mt);
    at += q.nb;
  }
  BT_CUDA(cudaGetLastError());
  // jobs: F~ per interface, series terms per (interface, level), nodes per level
  std::vector<int> top(S, 0);
  for (const TreeNode& nd : h->nodes) top[nd.m] = nd.level;
  std::vector<IfJob> jobs;
  auto blank = [] {
    IfJob j;
    j.a[0] = j.a[1] = -1;
    j.a_src[0] = j.a_src[1] = 0;
    j.b[0] = j.b[1] = 0;
    j.add_r = -1;
    j.sum_lev = 0;
    j.sum_lo = 0;
    j.sum_hi = -1;
    j.out_w = -1;
    j.out_c = -1;
    return j;
  };
  h->if_off.assign(1, 0);
  for (int s = 0; s < S; ++s) {
    IfJob j = blank();
    if (s > 0 && L > 1) {
      j.a[0] = s * L - 1;  // W_{k_s - 1}: last interior row of segment s-1
      j.b[0] = s;          // A_{k_s}
    }
    if (s * L + 1 < N && L > 1) {
      j.a[1] = s * L + 1;  // W_{k_s + 1}: first interior row of segment s
      j.b[1] = S + s;      // B_{k_s}
    }
    j.add_r = s * L;
    j.out_w = s * L;
    jobs.push_back(j);
  }
  h->if_off.push_back((int)jobs.size());
  for (int s = 0; s < S; ++s)
    for (int lev = 0; lev <= top[s]; ++lev) {
      IfJob j = blank();
      j.a[0] = s * L;                 // F~_s
      j.b[0] = 2 * S + lev * S + s;   // R[lev][s]
      j.out_c = lev * S + s;
      jobs.push_back(j);
    }
  h->if_off.push_back((int)jobs.size());
  for (int lev = 0; lev < depth; ++lev) {
    for (int q = h->level_off[lev]; q < h->level_off[lev + 1]; ++q) {
      const TreeNode& nd = h->nodes[q];
      IfJob j = blank();
      if (nd.l > 0) {
        j.a[0] = (nd.l - 1) * L;                 // X~_{l-1}
        j.b[0] = 2 * S + depth * S + nd.m;       // HL_m
      }
      if (nd.r < S - 1) {
        j.a[1] = (nd.r + 1) * L;                 // X~_{r+1}
        j.b[1] = 3 * S + depth * S + nd.m;       // HR_m
      }
      j.sum_lev = 0;  // the node's own slot of the node-sum buffer
      j.sum_lo = q;
      j.sum_hi = q;
      j.out_w = nd.m * L;
      jobs.push_back(j);
    }
    h->if_off.push_back((int)jobs.size());
  }
  // F~ of the forward / backward stage 2: W_{k_s + 1} is the residual panel's
  // row k_s + 1 (k_tc_fwd leaves it there), W_{k_s - 1} = y of the last row
  for (int s = 0; s < S; ++s) {
    IfJob j = jobs[h->if_off[0] + s];
    if (j.a[1] >= 0) j.a_src[1] = 1;
    jobs.push_back(j);
  }
  h->if_off.push_back((int)jobs.size());
  BT_TRY(h->arena.alloc(&h->if_jobs, jobs.size() * sizeof(IfJob)));
  BT_CUDA(cudaMemcpyAsync(h->if_jobs, jobs.data(), jobs.size() * sizeof(IfJob), cudaMemcpyHostToDevice, st));
  BT_CUDA(cudaStreamSynchronize(st));  // the host vector goes out of scope
  h->tc_if_bf16x3 = buf;
  return BT_OK;
}

template <class C>
size_t ifgemm_smem() {
  return 1024 + C::NA * C::SLOT + 2 * C::PT + kBars(C::NA, C::NP) * 8 + 16;
}

// Step 2.2 on the tensor cores (split BF16): F~, series terms, then one launch per level.
// fb: the forward / backward stage 2 (F~ reads W_{k_s+1} from the residual panel).
template <class CI>
bt_status run_interface_tc(bt_handle_s* h, const TcBuffers& tb, const int* done, int* status, cudaStream_t st,
                           bool fb = false) {
  using E = __nv_bfloat16;
  const int M = CI::M, N = (int)h->N, S = (int)h->S, Kp = (int)tb.Kp;
  BT_TRY(make_tc_interface(h, st));
  const int nblk = (4 + h->depth) * S;
  CUtensorMap tm_if, tm_w, tm_r;
  BT_TRY(make_map(&tm_if, h->tc_if_bf16x3, ET<E>::dt, CI::eb, (uint64_t)M, (uint64_t)CI::SP * nblk * M, CI::CE, M));
  BT_TRY(make_map(&tm_w, tb.w, ET<E>::dt, CI::eb, (uint64_t)M, (uint64_t)CI::SP * N * Kp, CI::CE, CI::NT));
  BT_TRY(make_map(&tm_r, tb.r, ET<E>::dt, CI::eb, (uint64_t)M, (uint64_t)CI::SP * N * Kp, CI::CE, CI::NT));
  const size_t smem = ifgemm_smem<CI>();
  BT_CUDA(cudaFuncSetAttribute(k_tc_ifgemm<E, CI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const IfJob* jobs = reinterpret_cast<const IfJob*>(h->if_jobs);
  const E* r = reinterpret_cast<const E*>(tb.r);
  E* w = reinterpret_cast<E*>(tb.w);
  // node sums of the series terms: [nodes][Kp][M] FP32 after the series terms
  const size_t tile = (size_t)Kp * M;
  const int nnodes = (int)h->nodes.size();
  float* csum = tb.c + (size_t)h->depth * S * tile;
  auto launch = [&](int g, const char* name, const float* sums) -> bt_status {
    const int j0 = h->if_off[g], nj = h->if_off[g + 1] - j0;
    if (nj <= 0) return BT_OK;
    ProfScope ps(h, st, name);
    k_tc_ifgemm<E, CI><<<dim3(Kp / CI::NT, nj), CI::THREADS, smem, st>>>(tm_if, tm_w, tm_r, jobs, j0, r, w, tb.c,
                                                                        sums, N, S, nblk, Kp, done, status);
    BT_CUDA(cudaGetLastError());
    return BT_OK;
  };
  BT_TRY(launch(fb ? 2 + h->depth : 0, "tc_iface", tb.c));
  BT_TRY(launch(1, "tc_iface", tb.c));
  {
    ProfScope ps(h, st, "tc_dichotomy");
    k_node_sums<<<dim3((unsigned)((tile + 1023) / 1024), nnodes), 256, 0, st>>>(tb.c, csum, h->d_nodes,
                                                                               h->d_mid_level, S, tile, done);
    BT_CUDA(cudaGetLastError());
  }
  for (int lev = 0; lev < h->depth; ++lev) BT_TRY(launch(2 + lev, "tc_dichotomy", csum));
  return BT_OK;
}

template <class C>
size_t sweep_smem() {
  return 1024 + C::NA * C::SLOT + (C::NP + C::YB) * C::PT + kBars(C::NA, C::NP) * 8 + 16;
}
template <class C>
size_t correct_smem() {
  const size_t staging = C::SW ? 0 : C::NP * C::PT + 2 * (size_t)C::NT * C::M * 4;
  return 1024 + C::NA * C::SLOT + 2 * C::PT + staging + kBars(C::NA, C::NP) * 8 + 16;
}

// CS: configuration of the sweep kernel, CC: of the correction kernel.
template <typename E, class CS, class CC>
bt_status run_tc(bt_handle_s* h, const TcBuffers& tb, int64_t K, double* X, int accumulate, const int* done,
                 int* status, cudaStream_t st) {
  constexpr int SP = CS::SP;
  static_assert(CS::SP == CC::SP, "one plane count per precision");
  const int M = CS::M, N = (int)h->N, L = (int)h->L, S = (int)h->S, Kp = (int)tb.Kp;
  CUtensorMap tm_fac_s, tm_fac_c, tm_r, tm_w, tm_wc, tm_d;
  // every CTA loads its own factor slices
  BT_TRY(make_map(&tm_fac_s, tb.fac, ET<E>::dt, CS::eb, (uint64_t)M, (uint64_t)SP * 5 * N * M, CS::CE, M));
  BT_TRY(make_map(&tm_fac_c, tb.fac, ET<E>::dt, CC::eb, (uint64_t)M, (uint64_t)SP * 5 * N * M, CC::CE, M));
  BT_TRY(make_map(&tm_r, tb.r, ET<E>::dt, CS::eb, (uint64_t)M, (uint64_t)SP * N * Kp, CS::CE, CS::NT));
  BT_TRY(make_map(&tm_w, tb.w, ET<E>::dt, CS::eb, (uint64_t)M, (uint64_t)SP * N * Kp, CS::CE, CS::NT));
  BT_TRY(make_map(&tm_wc, tb.w, ET<E>::dt, CC::eb, (uint64_t)M, (uint64_t)SP * N * Kp, CC::CE, CC::NT));
  // FP32 correction panel d, block-transposed like the work panel
  BT_TRY(make_map(&tm_d, tb.d, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (uint64_t)M, (uint64_t)N * Kp, 32, CC::NT));
  const E* r = reinterpret_cast<const E*>(tb.r);
  E* w = reinterpret_cast<E*>(tb.w);
  // unit stencils, split BF16, M = 128, results into a row-major FP32 panel:
  // forward pass, step 2.2, backward pass (no correction kernel)
  if constexpr (CS::SW && SP == 2 && M == 128 && std::is_same<E, __nv_bfloat16>::value) {
    if (accumulate == 2 && tb.drow != nullptr && h->stencil_unit && L > 1 && h->tc_fac_fb != nullptr) {
      using CF = CS;
      CUtensorMap tm_fb;
      BT_TRY(make_map(&tm_fb, h->tc_fac_fb, ET<E>::dt, CF::eb, (uint64_t)M, (uint64_t)SP * 4 * N * M, CF::CE, M));
      const size_t smem = 1024 + CF::NA * CF::SLOT + (CF::NP + 1) * CF::PT + (kBars(CF::NA, CF::NP) + 1) * 8 + 16;
      {
        BT_CUDA(cudaFuncSetAttribute(k_tc_fwd<CF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ProfScope ps(h, st, "tc_sweep");
        k_tc_fwd<CF><<<dim3(Kp / CF::NT, S), CF::THREADS, smem, st>>>(tm_fb, tm_r, tm_w, N, L, Kp, done, status);
        BT_CUDA(cudaGetLastError());
      }
      using CI = Cfg<E, CS::M, 128, 3, 2, 1, true>;
      BT_TRY(run_interface_tc<CI>(h, tb, done, status, st, true));
      {
        BT_CUDA(cudaFuncSetAttribute(k_tc_bwd<CF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ProfScope ps(h, st, "tc_correct");
        k_tc_bwd<CF><<<dim3(Kp / CF::NT, S), CF::THREADS, smem, st>>>(tm_fb, tm_w, (const E*)w, tb.drow, (int)K, N,
                                                                      L, S, Kp, done, status);
        BT_CUDA(cudaGetLastError());
      }
      return BT_OK;
    }
  }
  // step 2.1
  if (L > 1) {
    const size_t smem = sweep_smem<CS>();
    BT_CUDA(cudaFuncSetAttribute(k_tc_sweep<E, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(h, st, "tc_sweep");
    // A_i = I lets the forward sweep reuse Dinv_i for the recurrence term (needs a
    // ring that holds all of a block's slices plus one)
    const int shareD = (h->stencil && CS::NA > CS::NCH) ? 1 : 0;
    k_tc_sweep<E, CS><<<dim3(Kp / CS::NT, S), CS::THREADS, smem, st>>>(tm_fac_s, tm_r, tm_w, N, L, Kp, shareD, done,
                                                                       status);
  }
  BT_CUDA(cudaGetLastError());
  // step 2.2: tensor cores for the split-BF16 precision, FP32 CUDA cores otherwise
  if constexpr (SP == 2) {
    using CI = Cfg<E, CS::M, 128, 3, 2, 1, true>;
    BT_TRY(run_interface_tc<CI>(h, tb, done, status, st));
  } else {
    constexpr int KT = 32;   // columns per interface CTA
    constexpr int KD = 16;   // columns per dichotomy CTA (more CTAs on the narrow top levels)
    const TransposedF32& f = h->f32t;
    const size_t sm3 = 3 * (size_t)M * KT * sizeof(float);
    BT_CUDA(cudaFuncSetAttribute(k_tc_iface<E, SP, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
    {
      ProfScope ps(h, st, "tc_iface");
      k_tc_iface<E, SP, KT><<<dim3(S, Kp / KT), (M / 4) * (KT / 8), sm3, st>>>(r, w, f.AK, f.BK, f.R, h->d_mid_level,
                                                                            tb.c, N, M, S, L, Kp, done);
    }
    BT_CUDA(cudaGetLastError());
    for (int lev = 0; lev < h->depth; ++lev) {
      const int n0 = h->level_off[lev], nn = h->level_off[lev + 1] - n0;
      ProfScope ps(h, st, "tc_dichotomy");
      k_tc_dichotomy<E, SP, KD><<<dim3(nn, Kp / KD), (M / 4) * (KD / 8), 2 * (size_t)M * KD * sizeof(float), st>>>(
          w, tb.c, f.HL, f.HR, h->d_nodes, lev, n0, N, M, S, L, Kp, done);
    }
    BT_CUDA(cudaGetLastError());
  }
  // step 2.3
  {
    const int ntiles = Kp / CC::NT;
    const int rows = std::max(1, L - 1);
    int chunks = std::max(1, std::min(rows, (2 * 152 + S * ntiles - 1) / (S * ntiles)));
    const int rpc = (rows + chunks - 1) / chunks;
    chunks = (rows + rpc - 1) / rpc;
    if constexpr (CC::SW && CC::SP == 2 && CC::M == 128) {
      // interface tiles in TMEM, three factor slots, W rows through a two-stage
      // TMA ring (measured against seven slots with W read by the epilogue
      // threads: 1.27 against 1.70 ms per two corrections)
      using CT = Cfg<E, 128, 128, 3, 2, 2, true>;
      const size_t smem = 1024 + CT::NA * CT::SLOT + CT::NP * CT::PT + kBars(CT::NA, CT::NP) * 8 + 16;
      BT_CUDA(cudaFuncSetAttribute(k_tc_correct_ta<CT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      ProfScope ps(h, st, "tc_correct");
      // first solve: X = d written by the correction itself (no FP32 round trip)
      k_tc_correct_ta<CT, true><<<dim3(ntiles, S, chunks), CT::THREADS, smem, st>>>(
          tm_fac_c, tm_wc, (const E*)w, tb.d, (accumulate == 0 && h->M == CT::M) ? X : nullptr,
          accumulate == 2 ? tb.drow : nullptr,
          (int)K, N, L, S, Kp, L > 1 ? rpc : 0, done,
          status);
    } else {
      const size_t smem = correct_smem<CC>();
      BT_CUDA(cudaFuncSetAttribute(k_tc_correct<E, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      ProfScope ps(h, st, "tc_correct");
      k_tc_correct<E, CC><<<dim3(ntiles, S, chunks), CC::THREADS, smem, st>>>(
          tm_fac_c, tm_wc, tm_d, (const E*)w, tb.d, N, L, S, Kp, L > 1 ? rpc : 0, done, status);
    }
    BT_CUDA(cudaGetLastError());
    // the correction writes X itself in the first split-BF16 solve (M = 128, unpadded)
    const bool direct_x = CC::SW && CC::SP == 2 && CC::M == 128 && accumulate == 0 && h->M == CC::M;
    if (!direct_x && accumulate != 2) {
      const int Mr = (int)h->M;  // the true block size; the panel has M (= Mt) rows
      const int64_t nitem = (int64_t)((K + 31) / 32) * ((Mr + 7) / 8) * N;
      static const int grid = resident_grid(reinterpret_cast<const void*>(&k_x_update_warp), 256, 0);
      const int blocks = (int)std::min<int64_t>((nitem + 7) / 8, grid);
      ProfScope ps(h, st, "x_update");
      k_x_update_warp<<<blocks, 256, 0, st>>>(tb.d, X, N, Mr, M, (int)K, Kp, accumulate, done);
    }
  }
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

// sweep / correction configurations per (operand type, block size, planes)
// (sweep rings as deep as shared memory allows: a forward step consumes two
// blocks, so a ring of more than two blocks lets the next step's slices land
// while the current step waits for its recurrence operand)
using SwB128 = Cfg<__nv_bfloat16, 128, 64, 8, 1, 4>;
using CoB128 = Cfg<__nv_bfloat16, 128, 32, 6, 1, 4>;
using SwT128 = Cfg<float, 128, 32, 8, 1, 4>;
using CoT128 = Cfg<float, 128, 32, 6, 1, 4>;
using SwB64 = Cfg<__nv_bfloat16, 64, 128, 16, 1, 4>;
using CoB64 = Cfg<__nv_bfloat16, 64, 64, 8, 1, 4>;
using SwT64 = Cfg<float, 64, 64, 16, 1, 4>;
using CoT64 = Cfg<float, 64, 64, 8, 1, 4>;
using SwX128 = Cfg<__nv_bfloat16, 128, 128, 3, 2, 1, true>;
using CoX128 = Cfg<__nv_bfloat16, 128, 128, 3, 2, 1, true>;
using SwX64 = Cfg<__nv_bfloat16, 64, 64, 8, 2, 4>;
using CoX64 = Cfg<__nv_bfloat16, 64, 64, 6, 2, 4>;

}  // namespace

int tc_col_tile(int precision, int M) {
  (void)precision;
  // internal panels are padded to a multiple of every column tile in use
  return (M >= 1 && M <= 128) ? 128 : 0;
}

int tc_M(const bt_handle_s* h) { return h->M <= 64 ? 64 : h->M <= 128 ? 128 : 0; }

int tc_planes(int precision) { return precision == BT_PREC_BF16X3 ? 2 : 1; }

bt_status make_f32t_factors(bt_handle_s* h, cudaStream_t st) {
  TransposedF32& f = h->f32t;
  if (f.ready) return BT_OK;
  const int Mt = tc_M(h);
  const size_t MM = (size_t)Mt * Mt;
  struct Item {
    float** dst;
    const double* src;
    size_t nblk;
  } items[] = {{&f.AK, h->AK, (size_t)h->S}, {&f.BK, h->BK, (size_t)h->S}, {&f.R, h->R, (size_t)h->depth * h->S},
               {&f.HL, h->HL, (size_t)h->S}, {&f.HR, h->HR, (size_t)h->S}};
  for (auto& it : items) {
    BT_TRY(h->arena.alloc((void**)it.dst, it.nblk * MM * sizeof(float)));
    k_cast_transpose<<<512, 256, 0, st>>>(it.src, *it.dst, it.nblk, (int)h->M, Mt);
  }
  BT_CUDA(cudaGetLastError());
  f.ready = true;
  return BT_OK;
}

bt_status make_tc_factors(bt_handle_s* h, int precision, cudaStream_t st) {
  BT_TRY(make_f32t_factors(h, st));
  if (precision == BT_PREC_BF16X3 && h->M == 128 && h->stencil_unit && h->L > 1 && !h->tc_fac_fb) {
    // Dinv, G, Z = U^T, Y for the forward / backward stage 2 of unit stencils
    BT_TRY(factor_left_responses(h, st));
    const size_t nb = (size_t)h->N * h->M * h->M;
    void* buf = nullptr;
    BT_TRY(h->arena.alloc(&buf, (size_t)2 * 4 * nb * sizeof(__nv_bfloat16)));
    k_cast_fb<<<1024, 256, 0, st>>>(h->Dinv, h->G, h->U, h->Y, reinterpret_cast<__nv_bfloat16*>(buf), nb, (int)h->M);
    BT_CUDA(cudaGetLastError());
    h->tc_fac_fb = buf;
  }
  void** slot = precision == BT_PREC_BF16 ? &h->tc_fac_bf16 : precision == BT_PREC_TF32 ? &h->tc_fac_tf32 : &h->tc_fac_bf16x3;
  if (*slot) return BT_OK;
  const int Mt = tc_M(h), M = (int)h->M;
  const size_t nb = (size_t)h->N * Mt * Mt;
  const int sp = tc_planes(precision);
  const size_t eb = precision == BT_PREC_TF32 ? 4 : 2;
  BT_TRY(h->arena.alloc(slot, (size_t)sp * 5 * nb * eb));
  if (precision == BT_PREC_BF16)
    k_cast_factors<__nv_bfloat16, 1><<<1024, 256, 0, st>>>(h->Dinv, h->E, h->G, h->U, h->V,
                                                           reinterpret_cast<__nv_bfloat16*>(*slot), nb, M, Mt);
  else if (precision == BT_PREC_TF32)
    k_cast_factors<float, 1><<<1024, 256, 0, st>>>(h->Dinv, h->E, h->G, h->U, h->V, reinterpret_cast<float*>(*slot),
                                                   nb, M, Mt);
  else
    k_cast_factors<__nv_bfloat16, 2><<<1024, 256, 0, st>>>(h->Dinv, h->E, h->G, h->U, h->V,
                                                           reinterpret_cast<__nv_bfloat16*>(*slot), nb, M, Mt);
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

bt_status solve_tc(bt_handle_s* h, int precision, const TcBuffers& tb, int64_t K, double* X, int accumulate,
                   const int* done, int* status, cudaStream_t st) {
  const int M = tc_M(h);  // the block size, padded to the tile
  if (precision == BT_PREC_BF16) {
    if (M == 128) return run_tc<__nv_bfloat16, SwB128, CoB128>(h, tb, K, X, accumulate, done, status, st);
    if (M == 64) return run_tc<__nv_bfloat16, SwB64, CoB64>(h, tb, K, X, accumulate, done, status, st);
  } else if (precision == BT_PREC_TF32) {
    if (M == 128) return run_tc<float, SwT128, CoT128>(h, tb, K, X, accumulate, done, status, st);
    if (M == 64) return run_tc<float, SwT64, CoT64>(h, tb, K, X, accumulate, done, status, st);
  } else if (precision == BT_PREC_BF16X3) {
    if (M == 128) return run_tc<__nv_bfloat16, SwX128, CoX128>(h, tb, K, X, accumulate, done, status, st);
    if (M == 64) return run_tc<__nv_bfloat16, SwX64, CoX64>(h, tb, K, X, accumulate, done, status, st);
  }
  set_error("the tensor-core solve supports block sizes M <= 128");
  return BT_ERR_UNSUPPORTED;
}

}  // namespace bt
