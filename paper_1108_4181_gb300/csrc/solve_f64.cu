// Algorithm 2, stage 2 (Section 2.2, steps 2.1-2.3) in FP64.
//
// On GB300 the FP64 pipe issues about 2 fused multiply-adds per clock per SM
// (1.2 TFLOP/s for the chip), so these kernels are bound by FP64 issue, not by
// memory: a thread owns one row m of an M x kt output tile and CW of its
// columns, keeps CW independent accumulators, streams its block row from
// global memory (L1-resident within the loop) and reads the panel from shared
// memory as a broadcast.  Panels use the caller's layout (row-major
// (N*M) x K); blocks are row-major M x M.
//
// Kernels, one per step, launched back to back on one stream:
//   k_sweep      eq. sub3 per segment and column tile (step 2.1):
//                y_i = Dinv_i F_i + E_i y_{i-1}, then W_i = y_i + G_i W_{i+1};
//                W is written into X's interior rows.
//   k_iface      eq. red1 right-hand side F~_s = F_K + A_K W_{K-1} + B_K W_{K+1}
//                and the series terms c[l][s] = R[l][s] F~_s for every tree
//                level l at which interface s lies inside a node (step 2.2;
//                the dichotomy "reduces to the sum of a series", Section 1).
//   k_dichotomy  one launch per tree level (Algorithm 1, step 2.2):
//                X~_m = sum_{j in [l,r]} c[level][j] + HL_m X~_{l-1} + HR_m X~_{r+1},
//                written into X's interface row k_m.
//   k_correct    eq. superposition (step 2.3): X_i = W_i + U_i X~_s + V_i X~_{s+1}.

#include <algorithm>

#include "bt_internal.cuh"

namespace bt {

namespace {

struct F64Args {
  int64_t N, S, L, K;
  int M;
  const double *Dinv, *E, *G, *U, *V, *A, *B, *R, *HL, *HR;
  const int* nodes;
  const int* mid_level;
  double* c;  // [depth][S][M][K]
};

template <int CW>
__device__ __forceinline__ void acc_blk(double (&acc)[CW], const double* __restrict__ blk, int M, int m,
                                        const double* pan, int kt, int c0) {
  const double* row = blk + (size_t)m * M;
#pragma unroll 4
  for (int k = 0; k < M; ++k) {
    const double a = __ldg(row + k);
    const double* p = pan + k * kt + c0;
#pragma unroll
    for (int c = 0; c < CW; ++c) acc[c] = fma(a, p[c], acc[c]);
  }
}

// Stage an M x kt tile of a panel (row block at `src`, leading dimension K)
// into shared memory; columns at or beyond K read as zero.
__device__ __forceinline__ void load_tile(double* dst, const double* __restrict__ src, int M, int64_t K,
                                          int64_t col0, int kt) {
  for (int e = threadIdx.x; e < M * kt; e += blockDim.x) {
    const int r = e / kt, c = e % kt;
    const int64_t col = col0 + c;
    dst[e] = col < K ? src[(size_t)r * K + col] : 0.0;
  }
}

template <int CW>
__device__ __forceinline__ void load_own(double (&acc)[CW], const double* __restrict__ src, int m, int64_t K,
                                         int64_t col) {
#pragma unroll
  for (int c = 0; c < CW; ++c) acc[c] = (col + c < K) ? src[(size_t)m * K + col + c] : 0.0;
}

template <int CW>
__device__ __forceinline__ void store_own(const double (&acc)[CW], double* __restrict__ dst, int m, int64_t K,
                                          int64_t col) {
#pragma unroll
  for (int c = 0; c < CW; ++c)
    if (col + c < K) dst[(size_t)m * K + col + c] = acc[c];
}

template <int CW>
__global__ void k_sweep(F64Args p, const double* __restrict__ F, double* __restrict__ X) {
  extern __shared__ double sm[];
  const int M = p.M, CG = blockDim.x / M, kt = CW * CG;
  const int t = threadIdx.x, m = t / CG, c0 = (t % CG) * CW;
  const bool active = m < M;
  double* pf = sm;
  double* py = sm + M * kt;
  const int64_t s = blockIdx.x, col0 = (int64_t)blockIdx.y * kt, col = col0 + c0;
  const int64_t a = s * p.L + 1, b = s * p.L + p.L;
  const size_t MM = (size_t)M * M, MK = (size_t)M * p.K;
  // forward elimination: y_i = Dinv_i F_i + E_i y_{i-1}, y_{a-1} = W_{k_s} = 0
  for (int64_t i = a; i < b; ++i) {
    load_tile(pf, F + i * MK, M, p.K, col0, kt);
    __syncthreads();
    double acc[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) acc[c] = 0.0;
    if (active) {
      acc_blk<CW>(acc, p.Dinv + i * MM, M, m, pf, kt, c0);
      if (i > a) acc_blk<CW>(acc, p.E + i * MM, M, m, py, kt, c0);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < CW; ++c) py[m * kt + c0 + c] = acc[c];
      store_own<CW>(acc, X + i * MK, m, p.K, col);
    }
  }
  __syncthreads();
  // back substitution: W_{b-1} = y_{b-1}, W_i = y_i + G_i W_{i+1}, W_{k_s+L} = 0
  for (int64_t i = b - 2; i >= a; --i) {
    double acc[CW];
    if (active) {
      load_own<CW>(acc, X + i * MK, m, p.K, col);
      acc_blk<CW>(acc, p.G + i * MM, M, m, py, kt, c0);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < CW; ++c) py[m * kt + c0 + c] = acc[c];
      store_own<CW>(acc, X + i * MK, m, p.K, col);
    }
    __syncthreads();
  }
}

template <int CW>
__global__ void k_iface(F64Args p, const double* __restrict__ F, const double* __restrict__ X) {
  extern __shared__ double sm[];
  const int M = p.M, CG = blockDim.x / M, kt = CW * CG;
  const int t = threadIdx.x, m = t / CG, c0 = (t % CG) * CW;
  const bool active = m < M;
  double* pa = sm;
  double* pb = sm + M * kt;
  double* pt = sm + 2 * M * kt;
  const int64_t s = blockIdx.x, col0 = (int64_t)blockIdx.y * kt, col = col0 + c0;
  const int64_t Kr = s * p.L;
  const size_t MM = (size_t)M * M, MK = (size_t)M * p.K;
  const bool hasL = s > 0 && p.L > 1;       // W_{K-1}: last interior row of segment s-1
  const bool hasR = Kr + 1 < p.N && p.L > 1;  // W_{K+1}: first interior row of segment s
  if (hasL) load_tile(pa, X + (Kr - 1) * MK, M, p.K, col0, kt);
  if (hasR) load_tile(pb, X + (Kr + 1) * MK, M, p.K, col0, kt);
  __syncthreads();
  double acc[CW];
  if (active) {
    load_own<CW>(acc, F + Kr * MK, m, p.K, col);
    if (hasL) acc_blk<CW>(acc, p.A + Kr * MM, M, m, pa, kt, c0);
    if (hasR) acc_blk<CW>(acc, p.B + Kr * MM, M, m, pb, kt, c0);
#pragma unroll
    for (int c = 0; c < CW; ++c) pt[m * kt + c0 + c] = acc[c];
  }
  __syncthreads();
  if (!active) return;
  const int top = p.mid_level[s];
  for (int lev = 0; lev <= top; ++lev) {
    double cacc[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) cacc[c] = 0.0;
    acc_blk<CW>(cacc, p.R + ((size_t)lev * p.S + s) * MM, M, m, pt, kt, c0);
    store_own<CW>(cacc, p.c + ((size_t)lev * p.S + s) * MK, m, p.K, col);
  }
}

template <int CW>
__global__ void k_dichotomy(F64Args p, int lev, int node_off, double* __restrict__ X) {
  extern __shared__ double sm[];
  const int M = p.M, CG = blockDim.x / M, kt = CW * CG;
  const int t = threadIdx.x, m = t / CG, c0 = (t % CG) * CW;
  const bool active = m < M;
  double* pl = sm;
  double* pr = sm + M * kt;
  const int q = node_off + blockIdx.x;
  const int l = p.nodes[3 * q], r = p.nodes[3 * q + 1], mid = p.nodes[3 * q + 2];
  const int64_t col0 = (int64_t)blockIdx.y * kt, col = col0 + c0;
  const size_t MM = (size_t)M * M, MK = (size_t)M * p.K;
  const bool hl = l > 0, hr = r < p.S - 1;
  if (hl) load_tile(pl, X + (int64_t)(l - 1) * p.L * MK, M, p.K, col0, kt);
  if (hr) load_tile(pr, X + (int64_t)(r + 1) * p.L * MK, M, p.K, col0, kt);
  __syncthreads();
  if (!active) return;
  double acc[CW];
#pragma unroll
  for (int c = 0; c < CW; ++c) acc[c] = 0.0;
  for (int j = l; j <= r; ++j) {
    const double* cj = p.c + ((size_t)lev * p.S + j) * MK + (size_t)m * p.K + col;
#pragma unroll
    for (int c = 0; c < CW; ++c)
      if (col + c < p.K) acc[c] += cj[c];
  }
  if (hl) acc_blk<CW>(acc, p.HL + (size_t)mid * MM, M, m, pl, kt, c0);
  if (hr) acc_blk<CW>(acc, p.HR + (size_t)mid * MM, M, m, pr, kt, c0);
  store_own<CW>(acc, X + (int64_t)mid * p.L * MK, m, p.K, col);
}

template <int CW>
__global__ void k_correct(F64Args p, double* __restrict__ X, int rows_per_cta) {
  extern __shared__ double sm[];
  const int M = p.M, CG = blockDim.x / M, kt = CW * CG;
  const int t = threadIdx.x, m = t / CG, c0 = (t % CG) * CW;
  const bool active = m < M;
  double* p0 = sm;
  double* p1 = sm + M * kt;
  const int64_t s = blockIdx.x, col0 = (int64_t)blockIdx.y * kt, col = col0 + c0;
  const size_t MM = (size_t)M * M, MK = (size_t)M * p.K;
  const bool has_next = s + 1 < p.S;  // X~_S is the fictitious X_{N+1} = 0
  load_tile(p0, X + s * p.L * MK, M, p.K, col0, kt);
  if (has_next) load_tile(p1, X + (s + 1) * p.L * MK, M, p.K, col0, kt);
  __syncthreads();
  if (!active) return;
  const int64_t a = s * p.L + 1 + (int64_t)blockIdx.z * rows_per_cta;
  const int64_t b = std::min<int64_t>(a + rows_per_cta, s * p.L + p.L);
  for (int64_t i = a; i < b; ++i) {
    double acc[CW];
    load_own<CW>(acc, X + i * MK, m, p.K, col);
    acc_blk<CW>(acc, p.U + i * MM, M, m, p0, kt, c0);
    if (has_next) acc_blk<CW>(acc, p.V + i * MM, M, m, p1, kt, c0);
    store_own<CW>(acc, X + i * MK, m, p.K, col);
  }
}

template <int CW>
bt_status launch_all(bt_handle_s* h, F64Args a, const double* F, double* X, int CG, int stages,
                     cudaStream_t st) {
  const int M = a.M, kt = CW * CG, threads = M * CG;
  const int64_t ntiles = (a.K + kt - 1) / kt;
  if (ntiles > 65535 || a.S > 2147483647LL) {
    set_error("bt_solve: too many right-hand-side tiles for one launch");
    return BT_ERR_UNSUPPORTED;
  }
  const size_t sm2 = 2 * (size_t)M * kt * sizeof(double), sm3 = 3 * (size_t)M * kt * sizeof(double);
  if (sm3 > 48 * 1024) {
    for (const void* f : {(const void*)k_sweep<CW>, (const void*)k_iface<CW>, (const void*)k_dichotomy<CW>,
                          (const void*)k_correct<CW>})
      BT_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
  }
  if (a.L > 1) {
    ProfScope ps(h, st, "f64_sweep");
    k_sweep<CW><<<dim3((unsigned)a.S, (unsigned)ntiles), threads, sm2, st>>>(a, F, X);
    BT_CUDA(cudaGetLastError());
  }
  if (stages < 2) return BT_OK;
  {
    ProfScope ps(h, st, "f64_iface");
    k_iface<CW><<<dim3((unsigned)a.S, (unsigned)ntiles), threads, sm3, st>>>(a, F, X);
  }
  BT_CUDA(cudaGetLastError());
  for (int lev = 0; lev < h->depth; ++lev) {
    const int n0 = h->level_off[lev], nn = h->level_off[lev + 1] - n0;
    ProfScope ps(h, st, "f64_dichotomy");
    k_dichotomy<CW><<<dim3(nn, (unsigned)ntiles), threads, sm2, st>>>(a, lev, n0, X);
    BT_CUDA(cudaGetLastError());
  }
  if (stages < 3 || a.L < 2) return BT_OK;
  // enough CTAs to cover the GPU several times over
  const int64_t rows = a.L - 1;
  int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(rows, (4 * 152 + a.S * ntiles - 1) / (a.S * ntiles)));
  const int rows_per_cta = (int)((rows + chunks - 1) / chunks);
  chunks = (rows + rows_per_cta - 1) / rows_per_cta;
  {
    ProfScope ps(h, st, "f64_correct");
    k_correct<CW><<<dim3((unsigned)a.S, (unsigned)ntiles, (unsigned)chunks), threads, sm2, st>>>(a, X, rows_per_cta);
  }
  BT_CUDA(cudaGetLastError());
  return BT_OK;
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
    set_error(std::string("bt_solve: scratch allocation failed: ") + cudaGetErrorString(e));
    return BT_ERR_OOM;
  }
  h->scratch_bytes = bytes;
  return BT_OK;
}

bt_status solve_f64(bt_handle_s* h, const double* F, int64_t K, double* X, int stages, cudaStream_t st) {
  const int M = (int)h->M;
  BT_TRY(ensure_scratch(h, (size_t)h->depth * h->S * M * K * sizeof(double), st));
  F64Args a;
  a.N = h->N; a.S = h->S; a.L = h->L; a.K = K; a.M = M;
  a.Dinv = h->Dinv; a.E = h->E; a.G = h->G; a.U = h->U; a.V = h->V;
  a.A = h->A; a.B = h->B; a.R = h->R; a.HL = h->HL; a.HR = h->HR;
  a.nodes = h->d_nodes; a.mid_level = h->d_mid_level;
  a.c = reinterpret_cast<double*>(h->scratch);
  // column width per thread and column groups per CTA
  const int CW = K >= 4 ? 4 : (K >= 2 ? 2 : 1);
  int CG = (int)std::min<int64_t>((K + CW - 1) / CW, std::max(1, 128 / M));
  CG = std::max(1, std::min(CG, 1024 / M));
  switch (CW) {
    case 4: return launch_all<4>(h, a, F, X, CG, stages, st);
    case 2: return launch_all<2>(h, a, F, X, CG, stages, st);
    default: return launch_all<1>(h, a, F, X, CG, stages, st);
  }
}

}  // namespace bt
