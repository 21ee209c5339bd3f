// Algorithm 2, stage 2 (Section 2.2, steps 2.1-2.3) on the CUDA cores, for
// FP64 (the plain path) and FP32 (the SIMT low-precision solve used inside
// iterative refinement, and for the interface steps of the tensor-core path).
//
// On GB300 the FP64 pipe issues about 2 fused multiply-adds per clock per SM
// (1.2 TFLOP/s for the chip), so the FP64 kernels are bound by FP64 issue, not
// by memory: a thread owns one row m of an M x kt output tile and CW of its
// columns, keeps CW independent accumulators, streams its block row from
// global memory (L1-resident within the loop) and reads the panel from shared
// memory as a broadcast.  Panels use the caller's layout (row-major
// (N*M) x K); blocks are row-major M x M.
//
// Kernels, one per step, launched back to back on one stream:
//   k_sweep      eq. sub3 per segment and column tile (step 2.1):
//                y_i = Dinv_i F_i + E_i y_{i-1}, then W_i = y_i + G_i W_{i+1};
//                W is written into the work panel's interior rows.
//   k_iface      eq. red1 right-hand side F~_s = F_K + A_K W_{K-1} + B_K W_{K+1}
//                and the series terms c[l][s] = R[l][s] F~_s for every tree
//                level l at which interface s lies inside a node (step 2.2; the
//                dichotomy evaluation is a sum of a series over distributed
//                data, Section 1).
//   k_dichotomy  one launch per tree level (Algorithm 1, step 2.2):
//                X~_m = sum_{j in [l,r]} c[level][j] + HL_m X~_{l-1} + HR_m X~_{r+1},
//                written into the work panel's interface row k_m.
//   k_correct    eq. superposition (step 2.3): X_i = W_i + U_i X~_s + V_i X~_{s+1}.
// Every kernel returns at once when the refinement flag `done` is set.

#include <algorithm>
#include <cstddef>
#include <mutex>
#include <string>

#include "bt_internal.cuh"

namespace bt {

namespace {

template <typename T>
struct SimtArgs {
  int64_t N, S, L, K;
  int M;
  const T *Dinv, *E, *G, *U, *V, *AK, *BK, *R, *HL, *HR;
  const int* nodes;
  const int* mid_level;
  T* c;  // [depth][S][M][K]
  const int* done;
};

template <typename T>
__device__ __forceinline__ bool finished(const SimtArgs<T>& p) {
  return p.done != nullptr && *(volatile const int*)p.done != 0;
}

template <typename T, int CW>
__device__ __forceinline__ void acc_blk(T (&acc)[CW], const T* __restrict__ blk, int M, int m, const T* pan,
                                        int kt, int c0) {
  const T* row = blk + (size_t)m * M;
#pragma unroll 16
  for (int k = 0; k < M; ++k) {
    const T a = __ldg(row + k);
    const T* q = pan + k * kt + c0;
#pragma unroll
    for (int c = 0; c < CW; ++c) acc[c] = fma(a, q[c], acc[c]);
  }
}

// Stage an M x kt tile of a panel (row block at `src`, leading dimension K)
// into shared memory; columns at or beyond K read as zero.
// COH: read through L2 only (ld.global.cg).  The persistent batched kernel
// reads data that other CTAs wrote earlier in the same launch, which a
// non-coherent L1 line must not serve.
template <bool COH, typename T>
__device__ __forceinline__ T ld(const T* p) {
  if constexpr (COH) return __ldcg(p);
  return *p;
}

template <typename T, bool COH = false>
__device__ __forceinline__ void load_tile(T* dst, const T* __restrict__ src, int M, int64_t K, int64_t col0,
                                          int kt) {
  for (int e = threadIdx.x; e < M * kt; e += blockDim.x) {
    const int r = e / kt, c = e % kt;
    const int64_t col = col0 + c;
    dst[e] = col < K ? ld<COH>(src + (size_t)r * K + col) : T(0);
  }
}

template <typename T, typename U, int CW, bool COH = false>
__device__ __forceinline__ void load_own(T (&acc)[CW], const U* __restrict__ src, int m, int64_t K, int64_t col) {
#pragma unroll
  for (int c = 0; c < CW; ++c) acc[c] = (col + c < K) ? T(ld<COH>(src + (size_t)m * K + col + c)) : T(0);
}

template <typename T, typename U, int CW>
__device__ __forceinline__ void store_own(const T (&acc)[CW], U* __restrict__ dst, int m, int64_t K, int64_t col) {
#pragma unroll
  for (int c = 0; c < CW; ++c)
    if (col + c < K) dst[(size_t)m * K + col + c] = U(acc[c]);
}

// Each step is an item function over one (segment or node, column tile): the
// per-step kernels below run one item per CTA, the persistent batched kernel
// loops over a table of items.  An item starts with a barrier so that a CTA
// may run items back to back on the same shared memory.
template <typename T, int CW, bool COH = false>
__device__ __forceinline__ void sweep_item(const SimtArgs<T>& p, const T* __restrict__ Fin, T* __restrict__ Wk,
                                           int64_t s, int64_t tile, T* sm) {
  const int M = p.M, CG = blockDim.x / M, kt = CW * CG;
  const int t = threadIdx.x, m = t / CG, c0 = (t % CG) * CW;
  const bool active = m < M;
  T* pf = sm;
  T* py = sm + M * kt;
  const int64_t col0 = tile * kt, col = col0 + c0;
  __syncthreads();
  const int64_t a = s * p.L + 1, b = s * p.L + p.L;
  const size_t MM = (size_t)M * M, MK = (size_t)M * p.K;
  // forward elimination: y_i = Dinv_i F_i + E_i y_{i-1}, y_{a-1} = W_{k_s} = 0
  for (int64_t i = a; i < b; ++i) {
    load_tile<T, COH>(pf, Fin + i * MK, M, p.K, col0, kt);
    __syncthreads();
    T acc[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) acc[c] = T(0);
    if (active) {
      acc_blk<T, CW>(acc, p.Dinv + i * MM, M, m, pf, kt, c0);
      if (i > a) acc_blk<T, CW>(acc, p.E + i * MM, M, m, py, kt, c0);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < CW; ++c) py[m * kt + c0 + c] = acc[c];
      store_own<T, T, CW>(acc, Wk + i * MK, m, p.K, col);
    }
  }
  __syncthreads();
  // back substitution: W_{b-1} = y_{b-1}, W_i = y_i + G_i W_{i+1}, W_{k_s+L} = 0
  for (int64_t i = b - 2; i >= a; --i) {
    T acc[CW];
    if (active) {
      load_own<T, T, CW, COH>(acc, Wk + i * MK, m, p.K, col);
      acc_blk<T, CW>(acc, p.G + i * MM, M, m, py, kt, c0);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < CW; ++c) py[m * kt + c0 + c] = acc[c];
      store_own<T, T, CW>(acc, Wk + i * MK, m, p.K, col);
    }
    __syncthreads();
  }
}

template <typename T, int CW, bool COH = false>
__device__ __forceinline__ void iface_item(const SimtArgs<T>& p, const T* __restrict__ Fin,
                                           const T* __restrict__ Wk, int64_t s, int64_t tile, T* sm) {
  const int M = p.M, CG = blockDim.x / M, kt = CW * CG;
  const int t = threadIdx.x, m = t / CG, c0 = (t % CG) * CW;
  const bool active = m < M;
  T* pa = sm;
  T* pb = sm + M * kt;
  T* pt = sm + 2 * M * kt;
  const int64_t col0 = tile * kt, col = col0 + c0;
  __syncthreads();
  const int64_t Kr = s * p.L;
  const size_t MM = (size_t)M * M, MK = (size_t)M * p.K;
  const bool hasL = s > 0 && p.L > 1;         // W_{K-1}: last interior row of segment s-1
  const bool hasR = Kr + 1 < p.N && p.L > 1;  // W_{K+1}: first interior row of segment s
  if (hasL) load_tile<T, COH>(pa, Wk + (Kr - 1) * MK, M, p.K, col0, kt);
  if (hasR) load_tile<T, COH>(pb, Wk + (Kr + 1) * MK, M, p.K, col0, kt);
  __syncthreads();
  T acc[CW];
  if (active) {
    load_own<T, T, CW>(acc, Fin + Kr * MK, m, p.K, col);
    if (hasL) acc_blk<T, CW>(acc, p.AK + s * MM, M, m, pa, kt, c0);
    if (hasR) acc_blk<T, CW>(acc, p.BK + s * MM, M, m, pb, kt, c0);
#pragma unroll
    for (int c = 0; c < CW; ++c) pt[m * kt + c0 + c] = acc[c];
  }
  __syncthreads();
  if (!active) return;
  const int top = p.mid_level[s];
  for (int lev = 0; lev <= top; ++lev) {
    T cacc[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) cacc[c] = T(0);
    acc_blk<T, CW>(cacc, p.R + ((size_t)lev * p.S + s) * MM, M, m, pt, kt, c0);
    store_own<T, T, CW>(cacc, p.c + ((size_t)lev * p.S + s) * MK, m, p.K, col);
  }
}

// q: node index in the handle's node list (level `lev`).
template <typename T, int CW, bool COH = false>
__device__ __forceinline__ void dichotomy_item(const SimtArgs<T>& p, int lev, int q, T* __restrict__ Wk,
                                               int64_t tile, T* sm) {
  const int M = p.M, CG = blockDim.x / M, kt = CW * CG;
  const int t = threadIdx.x, m = t / CG, c0 = (t % CG) * CW;
  const bool active = m < M;
  T* pl = sm;
  T* pr = sm + M * kt;
  const int l = p.nodes[3 * q], r = p.nodes[3 * q + 1], mid = p.nodes[3 * q + 2];
  const int64_t col0 = tile * kt, col = col0 + c0;
  __syncthreads();
  const size_t MM = (size_t)M * M, MK = (size_t)M * p.K;
  const bool hl = l > 0, hr = r < p.S - 1;
  if (hl) load_tile<T, COH>(pl, Wk + (int64_t)(l - 1) * p.L * MK, M, p.K, col0, kt);
  if (hr) load_tile<T, COH>(pr, Wk + (int64_t)(r + 1) * p.L * MK, M, p.K, col0, kt);
  __syncthreads();
  if (!active) return;
  T acc[CW];
#pragma unroll
  for (int c = 0; c < CW; ++c) acc[c] = T(0);
#pragma unroll 8
  for (int j = l; j <= r; ++j) {
    const T* cj = p.c + ((size_t)lev * p.S + j) * MK + (size_t)m * p.K + col;
#pragma unroll
    for (int c = 0; c < CW; ++c)
      if (col + c < p.K) acc[c] += ld<COH>(cj + c);
  }
  if (hl) acc_blk<T, CW>(acc, p.HL + (size_t)mid * MM, M, m, pl, kt, c0);
  if (hr) acc_blk<T, CW>(acc, p.HR + (size_t)mid * MM, M, m, pr, kt, c0);
  store_own<T, T, CW>(acc, Wk + (int64_t)mid * p.L * MK, m, p.K, col);
}

// X_i = W_i + U_i X~_s + V_i X~_{s+1} on interior rows.  In place (Xout aliases
// the work panel, FP64 path) or into a separate FP64 panel, optionally added
// to its previous contents (refinement); in the separate case the interface
// rows receive X~_s as well.
template <typename T, int CW, bool COH = false>
__device__ __forceinline__ void correct_item(const SimtArgs<T>& p, const T* __restrict__ Wk,
                                             double* __restrict__ Xout, int64_t s, int64_t tile, int chunk,
                                             int rows_per_cta, int separate, int accumulate, T* sm) {
  const int M = p.M, CG = blockDim.x / M, kt = CW * CG;
  const int t = threadIdx.x, m = t / CG, c0 = (t % CG) * CW;
  const bool active = m < M;
  T* p0 = sm;
  T* p1 = sm + M * kt;
  const int64_t col0 = tile * kt, col = col0 + c0;
  __syncthreads();
  const size_t MM = (size_t)M * M, MK = (size_t)M * p.K;
  const bool has_next = s + 1 < p.S;  // X~_S is the fictitious X_{N+1} = 0
  load_tile<T, COH>(p0, Wk + s * p.L * MK, M, p.K, col0, kt);
  if (has_next) load_tile<T, COH>(p1, Wk + (s + 1) * p.L * MK, M, p.K, col0, kt);
  __syncthreads();
  if (!active) return;
  if (separate && chunk == 0) {
    T v[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) v[c] = p0[m * kt + c0 + c];
    double* xr = Xout + s * p.L * MK;
#pragma unroll
    for (int c = 0; c < CW; ++c)
      if (col + c < p.K) {
        double* o = xr + (size_t)m * p.K + col + c;
        *o = (accumulate ? *o : 0.0) + (double)v[c];
      }
  }
  const int64_t a = s * p.L + 1 + (int64_t)chunk * rows_per_cta;
  const int64_t b = std::min<int64_t>(a + rows_per_cta, s * p.L + p.L);
  for (int64_t i = a; i < b; ++i) {
    T acc[CW];
    load_own<T, T, CW, COH>(acc, Wk + i * MK, m, p.K, col);
    acc_blk<T, CW>(acc, p.U + i * MM, M, m, p0, kt, c0);
    if (has_next) acc_blk<T, CW>(acc, p.V + i * MM, M, m, p1, kt, c0);
    double* xr = Xout + i * MK;
#pragma unroll
    for (int c = 0; c < CW; ++c)
      if (col + c < p.K) {
        double* o = xr + (size_t)m * p.K + col + c;
        *o = ((separate && accumulate) ? *o : 0.0) + (double)acc[c];
      }
  }
}

template <typename T, int CW>
__global__ void k_sweep(SimtArgs<T> p, const T* __restrict__ Fin, T* __restrict__ Wk) {
  if (finished(p)) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  sweep_item<T, CW>(p, Fin, Wk, blockIdx.x, blockIdx.y, reinterpret_cast<T*>(smraw));
}

template <typename T, int CW>
__global__ void k_iface(SimtArgs<T> p, const T* __restrict__ Fin, const T* __restrict__ Wk) {
  if (finished(p)) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  iface_item<T, CW>(p, Fin, Wk, blockIdx.x, blockIdx.y, reinterpret_cast<T*>(smraw));
}

template <typename T, int CW>
__global__ void k_dichotomy(SimtArgs<T> p, int lev, int node_off, T* __restrict__ Wk) {
  if (finished(p)) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  dichotomy_item<T, CW>(p, lev, node_off + (int)blockIdx.x, Wk, blockIdx.y, reinterpret_cast<T*>(smraw));
}

template <typename T, int CW>
__global__ void k_correct(SimtArgs<T> p, const T* __restrict__ Wk, double* __restrict__ Xout, int rows_per_cta,
                          int separate, int accumulate) {
  if (finished(p)) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  correct_item<T, CW>(p, Wk, Xout, blockIdx.x, blockIdx.y, (int)blockIdx.z, rows_per_cta, separate, accumulate,
                      reinterpret_cast<T*>(smraw));
}

struct Plan {
  int CW, CG;
};

// FP64: issue-bound on the FP64 pipe; 4 columns per thread and about 128
// threads per CTA keep it busy.  FP32: 60x the FMA rate, so the factor
// stream becomes the bound; 8 columns per thread and up to 512 threads per
// CTA give each factor element fetched 16 to 64 uses.
template <typename T>
Plan pick_plan(int M, int64_t K) {
  Plan pl;
  const bool f32 = sizeof(T) == 4;
  pl.CW = (f32 && K >= 16) ? 16 : (f32 && K >= 8) ? 8 : (K >= 4 ? 4 : (K >= 2 ? 2 : 1));
  const int target = f32 ? 512 : 128;
  int CG = (int)std::min<int64_t>((K + pl.CW - 1) / pl.CW, std::max(1, target / M));
  pl.CG = std::max(1, std::min(CG, 1024 / M));
  return pl;
}

template <typename T, int CW>
bt_status launch_all(bt_handle_s* h, const SimtArgs<T>& a, const T* Fin, T* Wk, double* Xout, int CG, int stages,
                     int separate, int accumulate, cudaStream_t st, const char* tag) {
  const int M = a.M, kt = CW * CG, threads = M * CG;
  const int64_t ntiles = (a.K + kt - 1) / kt;
  if (ntiles > 65535) {
    set_error("bt_solve: too many right-hand-side tiles for one launch");
    return BT_ERR_UNSUPPORTED;
  }
  const size_t sm2 = 2 * (size_t)M * kt * sizeof(T), sm3 = 3 * (size_t)M * kt * sizeof(T);
  if (sm3 > 48 * 1024) {
    for (const void* f : {(const void*)k_sweep<T, CW>, (const void*)k_iface<T, CW>, (const void*)k_dichotomy<T, CW>,
                          (const void*)k_correct<T, CW>})
      BT_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
  }
  const bool f64 = sizeof(T) == 8;
  if (a.L > 1) {
    ProfScope ps(h, st, f64 ? "f64_sweep" : "f32_sweep");
    k_sweep<T, CW><<<dim3((unsigned)a.S, (unsigned)ntiles), threads, sm2, st>>>(a, Fin, Wk);
  }
  BT_CUDA(cudaGetLastError());
  if (stages < 2) return BT_OK;
  {
    ProfScope ps(h, st, f64 ? "f64_iface" : "f32_iface");
    k_iface<T, CW><<<dim3((unsigned)a.S, (unsigned)ntiles), threads, sm3, st>>>(a, Fin, Wk);
  }
  BT_CUDA(cudaGetLastError());
  for (int lev = 0; lev < h->depth; ++lev) {
    const int n0 = h->level_off[lev], nn = h->level_off[lev + 1] - n0;
    ProfScope ps(h, st, f64 ? "f64_dichotomy" : "f32_dichotomy");
    k_dichotomy<T, CW><<<dim3(nn, (unsigned)ntiles), threads, sm2, st>>>(a, lev, n0, Wk);
  }
  BT_CUDA(cudaGetLastError());
  if (stages < 3 || (a.L < 2 && !separate)) return BT_OK;
  // enough CTAs to cover the GPU several times over
  const int64_t rows = std::max<int64_t>(1, a.L - 1);
  int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(rows, (4 * 152 + a.S * ntiles - 1) / (a.S * ntiles)));
  const int rows_per_cta = (int)((rows + chunks - 1) / chunks);
  chunks = (rows + rows_per_cta - 1) / rows_per_cta;
  {
    ProfScope ps(h, st, f64 ? "f64_correct" : "f32_correct");
    k_correct<T, CW><<<dim3((unsigned)a.S, (unsigned)ntiles, (unsigned)chunks), threads, sm2, st>>>(
        a, Wk, Xout, rows_per_cta, separate, accumulate);
  }
  BT_CUDA(cudaGetLastError());
  (void)tag;
  return BT_OK;
}

template <typename T>
bt_status run(bt_handle_s* h, const SimtArgs<T>& a, const T* Fin, T* Wk, double* Xout, int stages, int separate,
              int accumulate, cudaStream_t st) {
  const Plan pl = pick_plan<T>(a.M, a.K);
  switch (pl.CW) {
    case 16: return launch_all<T, 16>(h, a, Fin, Wk, Xout, pl.CG, stages, separate, accumulate, st, "");
    case 8: return launch_all<T, 8>(h, a, Fin, Wk, Xout, pl.CG, stages, separate, accumulate, st, "");
    case 4: return launch_all<T, 4>(h, a, Fin, Wk, Xout, pl.CG, stages, separate, accumulate, st, "");
    case 2: return launch_all<T, 2>(h, a, Fin, Wk, Xout, pl.CG, stages, separate, accumulate, st, "");
    default: return launch_all<T, 1>(h, a, Fin, Wk, Xout, pl.CG, stages, separate, accumulate, st, "");
  }
}

}  // namespace

bt_status ensure_scratch(bt_handle_s* h, size_t bytes, cudaStream_t st) {
  if (bytes <= h->scratch_bytes) return BT_OK;
  if (h->scratch) {
    BT_CUDA(cudaStreamSynchronize(st));
    BT_CUDA(cudaFree(h->scratch));
    h->scratch = nullptr;
    h->scratch_bytes = 0;
  }
  cudaError_t e = cudaMalloc((void**)&h->scratch, bytes);
  if (e != cudaSuccess) {
    h->scratch = nullptr;
    set_error(std::string("bt_solve: scratch allocation failed: ") + cudaGetErrorString(e));
    return BT_ERR_OOM;
  }
  h->scratch_bytes = bytes;
  return BT_OK;
}

bt_status solve_f64(bt_handle_s* h, const double* F, int64_t K, double* X, int stages, cudaStream_t st) {
  const int M = (int)h->M;
  BT_TRY(ensure_scratch(h, (size_t)h->depth * h->S * M * K * sizeof(double), st));
  SimtArgs<double> a;
  a.N = h->N; a.S = h->S; a.L = h->L; a.K = K; a.M = M;
  a.Dinv = h->Dinv; a.E = h->E; a.G = h->G; a.U = h->U; a.V = h->V;
  a.AK = h->AK; a.BK = h->BK; a.R = h->R; a.HL = h->HL; a.HR = h->HR;
  a.nodes = h->d_nodes; a.mid_level = h->d_mid_level;
  a.c = reinterpret_cast<double*>(h->scratch);
  a.done = nullptr;
  return run<double>(h, a, F, X, X, stages, 0, 0, st);
}

bt_status solve_simt_f32(bt_handle_s* h, const float* r, int64_t K, float* d, float* c, double* X, int accumulate,
                         const int* done, cudaStream_t st) {
  const LowFactors& f = h->f32;
  SimtArgs<float> a;
  a.N = h->N; a.S = h->S; a.L = h->L; a.K = K; a.M = (int)h->M;
  a.Dinv = f.Dinv; a.E = f.E; a.G = f.G; a.U = f.U; a.V = f.V;
  a.AK = f.AK; a.BK = f.BK; a.R = f.R; a.HL = f.HL; a.HR = f.HR;
  a.nodes = h->d_nodes; a.mid_level = h->d_mid_level;
  a.c = c;
  a.done = done;
  return run<float>(h, a, r, d, X, 3, 1, accumulate, st);
}


}  // namespace bt

// ---------------------------------------------------------------------------
// Allocation-free FP64 solve (bt_solve_noalloc): the series-term scratch of
// the FP64 pipeline lives in a fixed array compiled into the library instead
// of the handle's grow-on-demand pool.  Host code must not take the array's
// name as a device address: its device address is looked up once per device
// with cudaGetSymbolAddress and handed to the kernels.
// ---------------------------------------------------------------------------
namespace bt {

static __device__ __align__(256) double g_noalloc_scratch[BT_NOALLOC_SCRATCH_BYTES / sizeof(double)];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
// Per device: the context the address was looked up in, and the address.  A
// device reset creates a new primary context in which the module (and the
// array) may sit elsewhere, so the address is looked up again when the
// current context differs from the recorded one.
struct NoAllocAddr {
  void* ctx;
  double* addr;
};
NoAllocAddr g_noalloc_addr[kNoAllocMaxDevices] = {};

// The current driver context (cuCtxGetCurrent through the runtime's driver
// entry point table; the library links only the runtime).
bool current_context(void** ctx) {
  using Fn = int (*)(void**);
  static Fn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (Fn) nullptr;
    return reinterpret_cast<Fn>(p);
  }();
  *ctx = nullptr;
  return fn != nullptr && fn(ctx) == 0 && *ctx != nullptr;
}
}  // namespace

bt_status solve_f64_noalloc(bt_handle_s* h, const double* F, int64_t K, double* X, cudaStream_t st) {
  // refuse before multiplying by K, so that a huge K cannot wrap the product
  const size_t per_col = (size_t)h->depth * h->S * h->M * sizeof(double);
  const size_t max_cols = per_col > 0 ? (size_t)BT_NOALLOC_SCRATCH_BYTES / per_col : 0;
  if (per_col == 0 || K <= 0 || (uint64_t)K > max_cols) {
    set_error("bt_solve_noalloc: needs depth*S*M*K*8 = " + std::to_string(per_col) + " * " + std::to_string(K) +
              " bytes of scratch, more than the " + std::to_string((size_t)BT_NOALLOC_SCRATCH_BYTES) +
              " bytes compiled into the library (at most K = " + std::to_string(max_cols) + " for this handle)");
    return BT_ERR_ARG;
  }
  int dev = 0;
  BT_CUDA(cudaGetDevice(&dev));
  if (dev != h->device || dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("bt_solve_noalloc: the handle's device must be current (and below device index 64)");
    return BT_ERR_ARG;
  }
  void* ctx = nullptr;
  if (!current_context(&ctx)) {
    set_error("bt_solve_noalloc: no current CUDA context on the handle's device");
    return BT_ERR_CUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocAddr& slot = g_noalloc_addr[dev];
    if (!slot.addr || slot.ctx != ctx) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "bt_solve_noalloc: cudaGetSymbolAddress");
      slot.addr = static_cast<double*>(p);
      slot.ctx = ctx;
    }
    scratch = slot.addr;
  }
  SimtArgs<double> a;
  a.N = h->N; a.S = h->S; a.L = h->L; a.K = K; a.M = (int)h->M;
  a.Dinv = h->Dinv; a.E = h->E; a.G = h->G; a.U = h->U; a.V = h->V;
  a.AK = h->AK; a.BK = h->BK; a.R = h->R; a.HL = h->HL; a.HR = h->HR;
  a.nodes = h->d_nodes; a.mid_level = h->d_mid_level;
  a.c = scratch;
  a.done = nullptr;
  return run<double>(h, a, F, X, X, 3, 0, 0, st);
}

}  // namespace bt

// ---------------------------------------------------------------------------
// Batched FP64 solve (bt_batch_*, bt_solve_batched; not in the paper): many
// right-hand-side sets, each against its own factored matrix, in ONE
// persistent cooperative launch.  The host builds a table of work items --
// (set, segment or node, column tile[, row chunk]) -- grouped into stages in
// the order of Algorithm 2's stage 2: sweeps, interface terms, one stage per
// dichotomy level, corrections.  Every CTA strides through a stage's items
// and meets the others at a grid barrier before the next stage; the barrier's
// wait is bounded (it records BT_ERR_TIMEOUT in the plan's status word and
// the kernel returns).  The whole launch is captured once into a CUDA graph.
// ---------------------------------------------------------------------------
namespace bt {

namespace {

struct BatchItem {
  int32_t set, a, tile, extra;  // a: segment or node; extra: row chunk or tree level
};

struct BatchSet {
  SimtArgs<double> p;
  const double* F;
  double* X;
  int32_t rows_per_cta;
};

enum : int32_t { kStSweep = 0, kStIface = 1, kStDich = 2, kStCorrect = 3 };

constexpr unsigned long long kBarrierLimitNs = 20ull * 1000000000ull;

// Control words of a plan (d_ctl, 64 bytes): [0] arrivals, [1] generation,
// [2] status -- cleared before every launch -- then, kept across launches,
// the barrier wait limit in ns at byte 16 (0: kBarrierLimitNs) and at byte 24
// a planted failure for tests: CTA 0 leaves the kernel instead of arriving at
// the barrier after that stage (-1: none).
struct BatchCtl {
  unsigned bar[2];
  int status;
  int pad;
  unsigned long long limit_ns;
  int skip_stage;
};
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sense-free grid barrier on two counters: bar[0] counts arrivals, bar[1] is
// the generation.  Returns false (after recording the failure) when the wait
// passes its time limit or another CTA has already failed.
__device__ bool grid_barrier(unsigned* bar, int* status, unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = gtimer();
      while (*gen == g) {
        if (*(volatile int*)status != 0 || gtimer() - t0 > limit_ns) {
          atomicCAS(status, 0, (int)BT_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <int CW>
__global__ void k_batched_f64(const BatchSet* __restrict__ sets, const BatchItem* __restrict__ items,
                              const int* __restrict__ stage_off, const int* __restrict__ stage_kind, int n_stages,
                              unsigned* bar, int* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* sm = reinterpret_cast<double*>(smraw);
  const BatchCtl* ctl = reinterpret_cast<const BatchCtl*>(bar);
  const unsigned long long lim = ctl->limit_ns ? ctl->limit_ns : kBarrierLimitNs;
  const int skip = ctl->skip_stage;
  for (int st = 0; st < n_stages; ++st) {
    const int kind = stage_kind[st];
    for (int i = stage_off[st] + (int)blockIdx.x; i < stage_off[st + 1]; i += (int)gridDim.x) {
      const BatchItem it = items[i];
      const BatchSet& B = sets[it.set];
      const SimtArgs<double> p = B.p;
      switch (kind) {
        case kStSweep: sweep_item<double, CW, true>(p, B.F, B.X, it.a, it.tile, sm); break;
        case kStIface: iface_item<double, CW, true>(p, B.F, B.X, it.a, it.tile, sm); break;
        case kStDich: dichotomy_item<double, CW, true>(p, it.extra, it.a, B.X, it.tile, sm); break;
        default:
          correct_item<double, CW, true>(p, B.X, B.X, it.a, it.tile, it.extra, B.rows_per_cta, 0, 0, sm);
          break;
      }
    }
    if (st + 1 < n_stages) {
      if (st == skip && blockIdx.x == 0) return;  // planted failure: this CTA never arrives
      if (!grid_barrier(bar, status, lim)) return;
    }
  }
}

template <int CW>
const void* batched_kernel() {
  return reinterpret_cast<const void*>(&k_batched_f64<CW>);
}

}  // namespace

bt_status batch_build(bt_batch_s* b, int32_t n, const bt_handle* hs, const double* const* F, const int64_t* K,
                      double* const* X, const bt_opts& o) {
  const int M = (int)hs[0]->M;
  int64_t kmax = 0;
  for (int i = 0; i < n; ++i) kmax = std::max(kmax, K[i]);
  b->CW = kmax >= 4 ? 4 : (kmax >= 2 ? 2 : 1);
  int CG = std::max(1, 128 / M);
  if (o.k_tile > 0) CG = std::max(1, o.k_tile / b->CW);
  CG = std::max(1, std::min(CG, 1024 / M));
  b->threads = M * CG;
  const int kt = b->CW * CG;
  b->k_tile = kt;
  b->smem = 3 * (size_t)M * kt * sizeof(double);

  // scratch for the series terms, one region per set (256-byte aligned)
  std::vector<size_t> coff(n);
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    coff[i] = total;
    total += ((size_t)hs[i]->depth * hs[i]->S * M * K[i] * sizeof(double) + 255) / 256 * 256;
  }
  if (total > 0) BT_TRY(b->arena.alloc((void**)&b->scratch, total));

  std::vector<BatchSet> sets(n);
  int max_depth = 0;
  bool any_interior = false;
  for (int i = 0; i < n; ++i) {
    const bt_handle_s* h = hs[i];
    SimtArgs<double>& a = sets[i].p;
    a.N = h->N; a.S = h->S; a.L = h->L; a.K = K[i]; a.M = M;
    a.Dinv = h->Dinv; a.E = h->E; a.G = h->G; a.U = h->U; a.V = h->V;
    a.AK = h->AK; a.BK = h->BK; a.R = h->R; a.HL = h->HL; a.HR = h->HR;
    a.nodes = h->d_nodes; a.mid_level = h->d_mid_level;
    a.c = reinterpret_cast<double*>(reinterpret_cast<char*>(b->scratch) + coff[i]);
    a.done = nullptr;
    sets[i].F = F[i];
    sets[i].X = X[i];
    // split each segment's interior rows so that the correction stage has
    // about as many items as the sweep has rows in flight
    const int64_t rows = std::max<int64_t>(1, h->L - 1);
    const int64_t chunks = std::min<int64_t>(rows, 4);
    sets[i].rows_per_cta = (int)((rows + chunks - 1) / chunks);
    max_depth = std::max(max_depth, h->depth);
    any_interior = any_interior || h->L > 1;
  }

  std::vector<BatchItem> items;
  std::vector<int> off{0}, kind;
  auto close_stage = [&](int k) {
    if ((int)items.size() > off.back()) {
      off.push_back((int)items.size());
      kind.push_back(k);
    }
  };
  auto tiles = [&](int i) { return (int32_t)((K[i] + kt - 1) / kt); };
  // item order: column tile fastest, so that neighbouring CTAs share factor blocks in L2
  if (any_interior) {
    for (int i = 0; i < n; ++i)
      if (hs[i]->L > 1)
        for (int32_t s = 0; s < hs[i]->S; ++s)
          for (int32_t t = 0; t < tiles(i); ++t) items.push_back({i, s, t, 0});
    close_stage(kStSweep);
  }
  for (int i = 0; i < n; ++i)
    for (int32_t s = 0; s < hs[i]->S; ++s)
      for (int32_t t = 0; t < tiles(i); ++t) items.push_back({i, s, t, 0});
  close_stage(kStIface);
  for (int lev = 0; lev < max_depth; ++lev) {
    for (int i = 0; i < n; ++i) {
      const bt_handle_s* h = hs[i];
      if (lev >= h->depth) continue;
      for (int q = h->level_off[lev]; q < h->level_off[lev + 1]; ++q)
        for (int32_t t = 0; t < tiles(i); ++t) items.push_back({i, q, t, lev});
    }
    close_stage(kStDich);
  }
  if (any_interior) {
    for (int i = 0; i < n; ++i) {
      const bt_handle_s* h = hs[i];
      if (h->L < 2) continue;
      const int64_t rows = h->L - 1;
      const int32_t chunks = (int32_t)((rows + sets[i].rows_per_cta - 1) / sets[i].rows_per_cta);
      for (int32_t c = 0; c < chunks; ++c)
        for (int32_t s = 0; s < h->S; ++s)
          for (int32_t t = 0; t < tiles(i); ++t) items.push_back({i, s, t, c});
    }
    close_stage(kStCorrect);
  }
  b->n_stages = (int)kind.size();
  b->n_items = (int64_t)items.size();

  BT_TRY(b->arena.alloc((void**)&b->d_sets, sets.size() * sizeof(BatchSet)));
  BT_TRY(b->arena.alloc((void**)&b->d_items, std::max<size_t>(1, items.size()) * sizeof(BatchItem)));
  BT_TRY(b->arena.alloc((void**)&b->d_stage_off, off.size() * sizeof(int)));
  BT_TRY(b->arena.alloc((void**)&b->d_stage_kind, std::max<size_t>(1, kind.size()) * sizeof(int)));
  BT_TRY(b->arena.alloc((void**)&b->d_ctl, 64));  // bar[2], status
  BT_CUDA(cudaMemcpy(b->d_sets, sets.data(), sets.size() * sizeof(BatchSet), cudaMemcpyHostToDevice));
  if (!items.empty())
    BT_CUDA(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
  BT_CUDA(cudaMemcpy(b->d_stage_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!kind.empty())
    BT_CUDA(cudaMemcpy(b->d_stage_kind, kind.data(), kind.size() * sizeof(int), cudaMemcpyHostToDevice));
  BT_CUDA(cudaMemset(b->d_ctl, 0, 64));
  const int no_skip = -1;
  BT_CUDA(cudaMemcpy(reinterpret_cast<char*>(b->d_ctl) + offsetof(BatchCtl, skip_stage), &no_skip, sizeof(int),
                     cudaMemcpyHostToDevice));

  const void* fn = b->CW == 4 ? batched_kernel<4>() : b->CW == 2 ? batched_kernel<2>() : batched_kernel<1>();
  b->kernel = fn;
  if (b->smem > 48 * 1024) BT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  int per_sm = 0, sms = 0;
  BT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, b->threads, b->smem));
  BT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  if (per_sm < 1) {
    set_error("bt_batch_create: the batched kernel does not fit on one SM");
    return BT_ERR_UNSUPPORTED;
  }
  b->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sms, std::max<int64_t>(1, b->n_items)));
  return BT_OK;
}

// Enqueues one batched solve on `st` (also used while capturing the graph).
bt_status batch_set_debug(bt_batch_s* b, unsigned long long limit_ns, int skip_stage) {
  BatchCtl c;
  BT_CUDA(cudaDeviceSynchronize());
  BT_CUDA(cudaMemcpy(&c, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost));
  c.limit_ns = limit_ns;
  c.skip_stage = skip_stage;
  BT_CUDA(cudaMemcpy(b->d_ctl, &c, sizeof(BatchCtl), cudaMemcpyHostToDevice));
  return BT_OK;
}

bt_status batch_enqueue(bt_batch_s* b, cudaStream_t st) {
  unsigned* bar = reinterpret_cast<unsigned*>(b->d_ctl);
  int* status = reinterpret_cast<int*>(b->d_ctl) + 2;
  BT_CUDA(cudaMemsetAsync(b->d_ctl, 0, 16, st));
  if (b->n_stages == 0) return BT_OK;
  const int n_stages = b->n_stages;
  void* args[] = {(void*)&b->d_sets, (void*)&b->d_items, (void*)&b->d_stage_off, (void*)&b->d_stage_kind,
                  (void*)&n_stages, (void*)&bar, (void*)&status};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)b->grid);
  cfg.blockDim = dim3((unsigned)b->threads);
  cfg.dynamicSmemBytes = b->smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BT_CUDA(cudaLaunchKernelExC(&cfg, b->kernel, args));
  return BT_OK;
}

}  // namespace bt
