// Algorithm 2, stage 1 (Section 2.2, steps 1.1-1.3) in FP64 on the GPU.
//
// The factorisation is a host-built schedule of two batched device
// primitives over M x M blocks:
//   GEMM: D[b] = alpha * X[b] Y[b] + beta * Z[b]
//   INV : Y[b] = X[b]^{-1}  (Gauss-Jordan with partial pivoting)
// Every operand address of every batch is computed on the host once, copied
// to the device in one transfer, and the primitives are launched in order on
// the caller's stream.
//
// Step 1.1, per segment (interior rows a = k_s+1 .. b = k_s+L-1, block sweep):
//   D_a = C_a,  D_i = C_i - A_i G_{i-1};   Dinv_i = D_i^{-1};
//   G_i = Dinv_i B_i (Gamma),  E_i = Dinv_i A_i;
//   V_b = G_b,  V_i = G_i V_{i+1}                    (eq. sub2: unit data at k_s+L)
//   Y_a = E_a,  Y_i = E_i Y_{i-1};  U_b = Y_b,  U_i = Y_i + G_i U_{i+1}
//                                                   (eq. sub1: unit data at k_s)
// Step 1.2, per interface K = k_s (eq. red1, U_0 = V_0 = 0):
//   At_s = A_K U_{K-1},  Ct_s = C_K - A_K V_{K-1} - B_K U_{K+1},  Bt_s = B_K V_{K+1}.
// Step 1.3, per node [l, r] with middle m of Algorithm 1 on P~ (rows of the
// inverse of the node's sub-matrix), from the Schur complements of its two
// sides:
//   left  DL_l = Ct_l,  DL_j = Ct_j - At_j DL_{j-1}^{-1} Bt_{j-1}       (j < m)
//   right DR_r = Ct_r,  DR_j = Ct_j - Bt_j DR_{j+1}^{-1} At_{j+1}       (j > m)
//   R_mm = (Ct_m - At_m DL_{m-1}^{-1} Bt_{m-1} - Bt_m DR_{m+1}^{-1} At_{m+1})^{-1}
//   R_mj = R_m,j+1 At_{j+1} DL_j^{-1} (j < m),  R_mj = R_m,j-1 Bt_{j-1} DR_j^{-1} (j > m)
//   HL = R_ml At_l (l > 0),  HR = R_mr Bt_r (r < S-1).
// The recurrences for R follow from R P_node = [0 .. I .. 0] column by column.

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>

#include <cooperative_groups.h>

#include "bt_internal.cuh"

namespace bt {

namespace {

// ---------------------------------------------------------------------------
// Batched FP64 GEMM on square M x M blocks: GT x GT output tile per CTA (GT =
// 64, 32 or 16), 256 threads with a (GT/16) x (GT/16) register tile each, K
// staged through shared memory 16 at a time.  The tile is chosen per M (see
// run_schedule).
// Operands come from a device table of pointers, 4 per batch entry: X, Y, Z
// (may be null when beta == 0), D (may alias Z).
// bp = (xlo, xhi, ylo, yhi) bounds the diagonals that may hold nonzeros:
// X[r][k] only where xlo <= k - r <= xhi, Y[k][c] only where ylo <= c - k <=
// yhi, for every matrix of the batch.  The contraction of a tile runs over the
// k that both bands admit for its rows and columns (a triangular or banded
// operand A_j, B_j halves or shortens it); the skipped terms are exact zeros,
// so the result is the same as the full contraction.  (-M, M, -M, M) = dense.
// ---------------------------------------------------------------------------
constexpr int GK = 16;

template <int GT>
__global__ void __launch_bounds__(256) k_gemm_batched(const double* const* __restrict__ tab, int M,
                                                      double alpha, double beta, int4 bp) {
  constexpr int R = GT / 16;  // register tile R x R
  const double* X = tab[4 * blockIdx.z + 0];
  const double* Y = tab[4 * blockIdx.z + 1];
  const double* Z = tab[4 * blockIdx.z + 2];
  double* D = const_cast<double*>(tab[4 * blockIdx.z + 3]);
  __shared__ double xs[GK][GT + 1];
  __shared__ double ys[GK][GT];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;
  const int kb = max(0, max(row0 + bp.x, col0 - bp.w)) / GK * GK;
  const int ke = min(M, min(row0 + GT + bp.y, col0 + GT - bp.z));
  for (int k0 = kb; k0 < ke; k0 += GK) {
    // X tile: rows row0..+GT, cols k0..+16 (stored transposed); Y tile: rows k0..+16, cols col0..+GT.
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      const int r = e / GK, c = e % GK;
      const int gr = row0 + r, gc = k0 + c;
      xs[c][r] = (gr < M && gc < M) ? X[(size_t)gr * M + gc] : 0.0;
      const int yr = k0 + e / GT, yc = col0 + e % GT;
      ys[e / GT][e % GT] = (yr < M && yc < M) ? Y[(size_t)yr * M + yc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double xv[R], yv[R];
#pragma unroll
      for (int i = 0; i < R; ++i) xv[i] = xs[kk][ty * R + i];
#pragma unroll
      for (int j = 0; j < R; ++j) yv[j] = ys[kk][tx * R + j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(xv[i], yv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int gr = row0 + ty * R + i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int gc = col0 + tx * R + j;
      if (gc >= M) continue;
      const size_t o = (size_t)gr * M + gc;
      double v = alpha * acc[i][j];
      if (beta != 0.0) v = fma(beta, Z[o], v);
      D[o] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Batched in-place Gauss-Jordan inversion with partial pivoting (row
// interchanges, undone as column interchanges at the end).  One CTA per
// matrix.  The matrix lives in shared memory when it fits, otherwise the CTA
// works directly on the output buffer in global memory (visibility between
// the CTA's threads is given by __syncthreads in both cases).
// tab: 2 pointers per batch entry, source and destination.
// A zero or non-finite pivot sets *status = 1 and is replaced by 1 so the
// remaining arithmetic stays finite.
// ---------------------------------------------------------------------------
constexpr int INV_SMEM_MAX = 160;  // M^2 doubles in shared memory up to this M

__global__ void __launch_bounds__(1024) k_inverse_batched(const double* const* __restrict__ tab, int M,
                                                          int use_smem, int* status) {
  extern __shared__ double sh[];
  const double* src = tab[2 * blockIdx.x + 0];
  double* dst = const_cast<double*>(tab[2 * blockIdx.x + 1]);
  double* a = use_smem ? sh : dst;
  double* fcol = use_smem ? sh + (size_t)M * M : sh;  // M multipliers
  int* perm = reinterpret_cast<int*>(fcol + M);       // M pivot rows
  __shared__ int s_piv;
  __shared__ double s_pval;
  const int nt = blockDim.x;
  const int MM = M * M;
  // elimination mapping: thread -> (row offset it0, column jt); rstep thread rows
  const int rstep = max(1, nt / M);
  const int jt = threadIdx.x < rstep * M ? threadIdx.x % M : M;
  const int it0 = threadIdx.x / M;
  for (int e = threadIdx.x; e < MM; e += nt) a[e] = src[e];
  __syncthreads();
  for (int k = 0; k < M; ++k) {
    // 1. pivot search over rows k..M-1 of column k (warp 0).
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + threadIdx.x; i < M; i += 32) {
        double v = fabs(a[(size_t)i * M + k]);
        if (v > best || (v == best && i < bi)) { best = v; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        double ob = __shfl_down_sync(0xffffffffu, best, off);
        int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        s_piv = bi;
        perm[k] = bi;
      }
    }
    __syncthreads();
    const int p = s_piv;
    // 2. row interchange k <-> p.
    if (p != k) {
      for (int j = threadIdx.x; j < M; j += nt) {
        double t = a[(size_t)k * M + j];
        a[(size_t)k * M + j] = a[(size_t)p * M + j];
        a[(size_t)p * M + j] = t;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double pv = a[(size_t)k * M + k];
      if (!(pv != 0.0) || !isfinite(pv)) {
        atomicExch(status, 1);
        pv = 1.0;
      }
      s_pval = pv;
    }
    // multipliers of column k (rows other than k are not touched by step 3)
    for (int i = threadIdx.x; i < M; i += nt) fcol[i] = (i == k) ? 0.0 : a[(size_t)i * M + k];
    __syncthreads();
    // 3. scale the pivot row; the pivot column entry becomes 1/pivot.
    const double pv = s_pval;
    for (int j = threadIdx.x; j < M; j += nt) {
      double v = (j == k) ? 1.0 : a[(size_t)k * M + j];
      a[(size_t)k * M + j] = v / pv;
    }
    __syncthreads();
    // 4. eliminate column k from every other row: thread -> column j (fixed),
    //    rows strided by the number of thread rows (no per-element division).
    if (jt < M) {
      const double pk = a[(size_t)k * M + jt];
      for (int i = it0; i < M; i += rstep) {
        if (i == k) continue;
        const size_t e = (size_t)i * M + jt;
        const double base = (jt == k) ? 0.0 : a[e];
        a[e] = fma(-fcol[i], pk, base);
      }
    }
    __syncthreads();
  }
  // undo the interchanges as column swaps, last first
  for (int k = M - 1; k >= 0; --k) {
    int p = perm[k];
    if (p != k) {
      for (int i = threadIdx.x; i < M; i += nt) {
        double t = a[(size_t)i * M + k];
        a[(size_t)i * M + k] = a[(size_t)i * M + p];
        a[(size_t)i * M + p] = t;
      }
    }
    __syncthreads();
  }
  if (use_smem)
    for (int e = threadIdx.x; e < MM; e += nt) dst[e] = a[e];
}

// ---------------------------------------------------------------------------
// The same Gauss-Jordan inversion on a thread-block cluster of C CTAs per
// matrix (C = 2, 4 or 8, chosen at launch), M <= 256.  CTA r holds columns
// [r Mc, (r+1) Mc) (Mc = ceil(M / C)) column-major in its shared memory, and
// each warp owns whole columns: the interchange of rows k and p and the
// elimination touch only a warp's own columns, so within a step no warp
// waits for another.  Row scaling is deferred: the stored rows keep their
// raw values U and row k records s_k = 1 / pivot; the inverse is s_i U[i][j]
// (rows scaled on the way out).  With g_i = U[i][k] / pivot (after the
// interchange), step k is
//   U[i][j] -= g_i U[k][j]      (i != k, j != k)
//   U[i][k]  = -g_i             (i != k),   U[k][k] = 1,
// the GJ step on s U.  The warp owning column k+1 updates it first, picks the
// pivot of step k+1 (the largest |U[i][k+1]|, i > k; ties to the lower row),
// forms 1 / pivot (an FP32 seed and two Newton-Raphson steps in FP64, four
// dependent FP64 operations) and writes p, 1 / pivot and the multipliers g
// into every CTA's shared memory (double-buffered by the parity of the step).
// One cluster barrier per step, split: a warp arrives as soon as it has read
// the step's pivot data (the publishing warp after publishing) and waits at
// the start of the next step, so the pivot chain runs ahead of the bulk of
// the elimination.  The interchanges are undone at the end by writing column
// c of the result to the column the composed interchanges send it to.
// Singular or non-finite pivots: as above.
// ---------------------------------------------------------------------------

// 1 / v for finite nonzero v: the FP32 reciprocal of v's leading significand
// bits (exponent from the bits) as the seed, then two Newton-Raphson steps
// r <- r + r (1 - v r) in FP64 (error about 2^-24 -> 2^-48 -> rounding);
// a division outside the normal range.
__device__ __forceinline__ double recip_newton(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7FF);
  if (be < 4 || be > 2042) return 1.0 / v;
  const float m = __uint_as_float(0x3F800000u | (unsigned)((b >> 29) & 0x7FFFFFu));  // [1, 2)
  const unsigned rb = __float_as_uint(1.0f / m);                                     // (0.5, 1]
  const int re = (int)((rb >> 23) & 0xFF) - 127 - (be - 1023) + 1023;
  double r = __longlong_as_double((long long)((b & 0x8000000000000000ull) | ((unsigned long long)re << 52) |
                                              ((unsigned long long)(rb & 0x7FFFFFu) << 29)));
  double e = fma(-v, r, 1.0);
  r = fma(r, e, r);
  e = fma(-v, r, 1.0);
  return fma(r, e, r);
}

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

constexpr int kInvClusterMaxM = 256;  // 8 rows per lane

__global__ void __launch_bounds__(1024) k_inverse_cluster(const double* const* __restrict__ tab, int M, int* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double sh[];
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int mat = blockIdx.x / C;
  const double* src = tab[2 * mat + 0];
  double* dst = const_cast<double*>(tab[2 * mat + 1]);
  const int Mc = (M + C - 1) / C;
  const int c0 = rank * Mc, nc = max(0, min(Mc, M - c0));  // global columns c0 .. c0 + nc - 1
  const int ldu = M | 1;                                   // column stride (odd: the transposing load spreads banks)
  double* U = sh;                                          // [Mc][ldu]: local column j, row i
  double* gbuf = U + (((size_t)Mc * ldu + 1) & ~(size_t)1);  // [2][M] multipliers (16-byte aligned)
  double* rbuf = gbuf + 2 * M;                             // [2] 1 / pivot
  double* srow = rbuf + 2;                                 // [M] row scales
  int* pbuf = reinterpret_cast<int*>(srow + M);            // [2] pivot rows
  int* perm = pbuf + 2;                                    // [M]
  int* pos = perm + M;                                     // [M]
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  for (int e = tid; e < M * Mc; e += nt) {
    const int i = e / Mc, lc = e % Mc;
    U[(size_t)lc * ldu + i] = lc < nc ? src[(size_t)i * M + c0 + lc] : 0.0;
  }
  __syncthreads();
  cl.sync();  // every CTA of the cluster runs before any shared memory is written remotely
  // The warp owning column kk (updated through step kk-1): pivot of step kk.
  auto pivot_col = [&](int kk, int slot) {
    const double* col = U + (size_t)(kk - c0) * ldu;
    unsigned long long bb = 0;
    int bi = 0x7fffffff;
    for (int i = kk + lane; i < M; i += 32) {
      const unsigned long long u = (unsigned long long)__double_as_longlong(col[i]) & 0x7FFFFFFFFFFFFFFFull;
      if (u > bb || bi == 0x7fffffff) {
        bb = u;
        bi = i;
      }
    }
    // the warp's largest 64-bit key, then the lowest row holding it: three reductions
    const unsigned kh = (unsigned)(bb >> 32), kl = (unsigned)bb;
    const unsigned mh = __reduce_max_sync(0xffffffffu, bi != 0x7fffffff ? kh : 0u);
    const unsigned ml = __reduce_max_sync(0xffffffffu, (bi != 0x7fffffff && kh == mh) ? kl : 0u);
    const int p = (int)__reduce_min_sync(0xffffffffu, (bi != 0x7fffffff && kh == mh && kl == ml) ? (unsigned)bi
                                                                                                : 0x7fffffffu);
    const double xp = col[p], xk = col[kk];
    double rinv = 0.0;
    if (lane == 0) {
      double pv = xp;
      if (!(pv != 0.0) || !isfinite(pv)) {
        atomicExch(status, 1);
        pv = 1.0;
      }
      rinv = recip_newton(pv);
    }
    rinv = __shfl_sync(0xffffffffu, rinv, 0);
    if ((M & 1) == 0) {  // rows in pairs: 16-byte stores
      for (int i = 2 * lane; i < M; i += 64) {
        const double2 gi = make_double2((i == p ? xk : col[i]) * rinv, (i + 1 == p ? xk : col[i + 1]) * rinv);
        for (int r = 0; r < C; ++r) {
          double* gr = r == rank ? gbuf : cl.map_shared_rank(gbuf, r);
          *reinterpret_cast<double2*>(gr + slot * M + i) = gi;
        }
      }
    } else {
      for (int i = lane; i < M; i += 32) {
        const double gi = (i == p ? xk : col[i]) * rinv;
        for (int r = 0; r < C; ++r) {
          if (r == rank)
            gbuf[slot * M + i] = gi;
          else
            cl.map_shared_rank(gbuf, r)[slot * M + i] = gi;
        }
      }
    }
    if (lane < C) {
      cl.map_shared_rank(pbuf, lane)[slot] = p;
      cl.map_shared_rank(rbuf, lane)[slot] = rinv;
    }
  };
  if (rank == 0 && w == 0) pivot_col(0, 0);
  cluster_arrive();
  for (int k = 0; k < M; ++k) {
    cluster_wait();  // the pivot of step k is published
    const int b = k & 1;
    const int p = pbuf[b];
    const double* g = gbuf + b * M;
    if (tid == 0) {
      perm[k] = p;
      srow[k] = rbuf[b];
    }
    const int owner = k / Mc, lk = k - owner * Mc;
    const int kn = k + 1;
    const int jn = (kn < M && kn / Mc == rank && (kn - c0) % nw == w) ? kn - c0 : -1;  // this warp's next pivot column
    double gv[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int i = lane + 32 * m;
      gv[m] = i < M ? g[i] : 0.0;
    }
    if (jn < 0) cluster_arrive();  // everything of step k is read
    // this warp's columns, the next pivot column first
    for (int t = -1; t * nw + w < Mc; ++t) {
      int j;
      if (t < 0) {
        if (jn < 0) continue;
        j = jn;
      } else {
        j = t * nw + w;
        if (j == jn) continue;
      }
      double* col = U + (size_t)j * ldu;
      const double vp = col[p], vk = col[k];
      __syncwarp();
      if (rank == owner && j == lk) {
        // column k of the inverse: -g, and 1 in row k (whose scale is 1 / pivot)
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int i = lane + 32 * m;
          if (i < M) col[i] = i == k ? 1.0 : __longlong_as_double(__double_as_longlong(gv[m]) ^ (long long)(1ULL << 63));
        }
      } else {
        // rows k and p interchanged: row k takes row p (vp), row p row k (vk)
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int i = lane + 32 * m;
          if (i < M) {
            const double v = fma(-gv[m], vp, i == p ? vk : col[i]);
            col[i] = i == k ? vp : v;
          }
        }
      }
      __syncwarp();
      if (t < 0) {
        pivot_col(kn, b ^ 1);
        cluster_arrive();
      }
    }
  }
  cluster_wait();
  // the interchanges undone as column interchanges, last first: position j
  // ends up holding elimination column pos[j]; column c goes to perm[c]
  if (tid == 0) {
    for (int c = 0; c < M; ++c) pos[c] = c;
    for (int k = M - 1; k >= 0; --k) {
      const int q = perm[k];
      const int t = pos[k];
      pos[k] = pos[q];
      pos[q] = t;
    }
    for (int j = 0; j < M; ++j) perm[pos[j]] = j;
  }
  __syncthreads();
  for (int e = tid; e < M * nc; e += nt) {
    const int i = e / nc, lc = e % nc;
    dst[(size_t)i * M + perm[c0 + lc]] = srow[i] * U[(size_t)lc * ldu + i];
  }
  cl.sync();  // no CTA leaves while a partner may still write into its shared memory
}

// Shared memory and threads of k_inverse_cluster for block size M on clusters of C CTAs.
size_t inv_cluster_smem(int M, int C) {
  const size_t Mc = (size_t)(M + C - 1) / C, ldu = (size_t)(M | 1);
  return (Mc * ldu + 1 + 3 * (size_t)M + 2) * sizeof(double) + (2 + 2 * (size_t)M) * sizeof(int);
}
int inv_cluster_threads(int M, int C) { return 32 * std::min(32, (M + C - 1) / C); }

// Plain device copy (grid-stride).
__global__ void k_copy(const double* __restrict__ src, double* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// dst[s] = src[s * L] for s < S (blocks of MM doubles).
__global__ void k_gather_blocks(const double* __restrict__ src, double* __restrict__ dst, int64_t S, int64_t L,
                                size_t MM) {
  const size_t n = (size_t)S * MM;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t s = e / MM, o = e % MM;
    dst[e] = src[s * L * MM + o];
  }
}

// Cdiag[j][m] = (C_j[m][m-1], C_j[m][m], C_j[m][m+1]), zero outside the block;
// Cdw[j][m] = C_j[m][m] as two FP32 terms (the rounded value, then the rounded
// remainder).  *not_unit is set when an off-diagonal inside a block is not
// exactly -1 or a diagonal entry lies outside [2^-30, 2^30] in magnitude.
__global__ void k_tridiag(const double* __restrict__ C, double* __restrict__ Cd, float* __restrict__ Cdw,
                          int64_t N, int M, int* not_unit) {
  const size_t n = (size_t)N * M;
  bool bad = false;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t j = e / M;
    const int m = (int)(e % M);
    const double* Cj = C + j * (size_t)M * M + (size_t)m * M;
    const double lo = m > 0 ? Cj[m - 1] : 0.0, d = Cj[m], up = m + 1 < M ? Cj[m + 1] : 0.0;
    Cd[3 * e + 0] = lo;
    Cd[3 * e + 1] = d;
    Cd[3 * e + 2] = up;
    const float dh = __double2float_rn(d);
    Cdw[2 * e] = dh;
    Cdw[2 * e + 1] = __double2float_rn(d - (double)dh);
    const double ad = fabs(d);
    bad = bad || (m > 0 && lo != -1.0) || (m + 1 < M && up != -1.0) || !(ad >= 0x1p-30 && ad <= 0x1p30);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(not_unit, 1);
}

__global__ void k_set_identity(double* I, int M) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * M; e += gridDim.x * blockDim.x)
    I[e] = (e / M == e % M) ? 1.0 : 0.0;
}

// Stencil detection: A_j = B_j = I (where used) and C_j tridiagonal.  A
// thread stops at its first violation and leaves the scan once another has
// reported one; each warp reports with one vote and one atomic (a dense
// operator fails almost everywhere, and one atomic per element serialised).
__global__ void k_detect_stencil(const double* A, const double* B, const double* C, int64_t N, int M,
                                 int* not_stencil) {
  const size_t n = (size_t)N * M * M;
  bool bad = false;
  int poll = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t j = e / ((size_t)M * M);
    const int r = (e / M) % M, c = e % M;
    const double id = (r == c) ? 1.0 : 0.0;
    if ((j > 0 && A[e] != id) || (j < N - 1 && B[e] != id) || ((c > r + 1 || r > c + 1) && C[e] != 0.0)) {
      bad = true;
      break;
    }
    if ((++poll & 15) == 0 && *(volatile const int*)not_stencil != 0) break;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(not_stencil, 1);
}

// Diagonal bands of the coupling blocks: the smallest and largest c - r over
// the nonzero (or non-finite) entries (r, c) of A_j, j >= 1, into prof[0..1]
// and of B_j, j <= N - 2, into prof[2..3] (prof preset to INT_MAX, INT_MIN).
// A block matrix made from a band matrix of half-bandwidths kl, ku <= M has
// upper triangular A_j (c - r >= M - kl) and lower triangular B_j.
__global__ void k_band_profile(const double* A, const double* B, int64_t N, int M, int* prof) {
  const size_t MM = (size_t)M * M, n = (size_t)N * MM;
  int alo = INT_MAX, ahi = INT_MIN, blo = INT_MAX, bhi = INT_MIN;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t j = (int64_t)(e / MM);
    const size_t w = e - (size_t)j * MM;
    const int d = (int)(w % M) - (int)(w / M);
    const double a = A[e], b = B[e];
    if (j > 0 && a != 0.0) { alo = min(alo, d); ahi = max(ahi, d); }
    if (j < N - 1 && b != 0.0) { blo = min(blo, d); bhi = max(bhi, d); }
  }
  alo = __reduce_min_sync(0xffffffffu, alo);
  ahi = __reduce_max_sync(0xffffffffu, ahi);
  blo = __reduce_min_sync(0xffffffffu, blo);
  bhi = __reduce_max_sync(0xffffffffu, bhi);
  if ((threadIdx.x & 31) == 0) {
    if (alo <= ahi) { atomicMin(prof + 0, alo); atomicMax(prof + 1, ahi); }
    if (blo <= bhi) { atomicMin(prof + 2, blo); atomicMax(prof + 3, bhi); }
  }
}

// D_e = X_e for every batch entry (pairs of block pointers), 4 values a thread.
__global__ void k_copy_blocks(const double* const* __restrict__ tab, size_t MM) {
  const double* X = tab[2 * blockIdx.y];
  double* D = const_cast<double*>(tab[2 * blockIdx.y + 1]);
  const size_t i0 = (size_t)blockIdx.x * 1024 + threadIdx.x;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const size_t i = i0 + (size_t)u * 256;
    if (i < MM) D[i] = X[i];
  }
}

// ---------------------------------------------------------------------------
// Schedule builder
// ---------------------------------------------------------------------------
struct Op {
  int kind;  // 0 = GEMM, 1 = INV, 2 = join (lane 0 waits for lane 1), 3 = copy
  int batch;
  size_t off;  // into the pointer table
  double alpha, beta;
  int4 bp;     // operand bands of a GEMM (see k_gemm_batched)
  int lane;    // 0: the caller's stream; 1: a second, lower-priority stream
               // that runs beside lane 0 and first waits for everything
               // enqueued on lane 0 before it
};

struct Schedule {
  std::vector<const double*> tab;
  std::vector<Op> ops;
  // The identity block: a product X I with alpha = 1 and no Z is the copy
  // D = X (exact on every path; the digit-slice products could not balance
  // the contraction index of such a product against X's column scales)
  const double* ident = nullptr;
  // GEMM batch under construction
  void gemm(double alpha, double beta, int4 bp, const std::vector<const double*>& X,
            const std::vector<const double*>& Y, const std::vector<const double*>& Z,
            const std::vector<double*>& D, int lane = 0) {
    if (D.empty()) return;
    std::vector<size_t> prod, copy;
    for (size_t b = 0; b < D.size(); ++b)
      (ident && Y[b] == ident && alpha == 1.0 && (beta == 0.0 || Z.empty() || !Z[b]) ? copy : prod).push_back(b);
    if (!copy.empty()) {
      Op o{3, (int)copy.size(), tab.size(), 0.0, 0.0, make_int4(0, 0, 0, 0), lane};
      for (size_t b : copy) {
        tab.push_back(X[b]);
        tab.push_back(D[b]);
      }
      ops.push_back(o);
    }
    if (prod.empty()) return;
    Op o{0, (int)prod.size(), tab.size(), alpha, beta, bp, lane};
    for (size_t b : prod) {
      tab.push_back(X[b]);
      tab.push_back(Y[b]);
      tab.push_back(Z.empty() ? nullptr : Z[b]);
      tab.push_back(D[b]);
    }
    ops.push_back(o);
  }
  void inv(const std::vector<const double*>& X, const std::vector<double*>& Y) {
    if (Y.empty()) return;
    Op o{1, (int)Y.size(), tab.size(), 0.0, 0.0, make_int4(0, 0, 0, 0), 0};
    for (size_t b = 0; b < Y.size(); ++b) {
      tab.push_back(X[b]);
      tab.push_back(Y[b]);
    }
    ops.push_back(o);
  }
  void join() { ops.push_back(Op{2, 0, 0, 0.0, 0.0, make_int4(0, 0, 0, 0), 0}); }
};

// Helper collecting one batched GEMM entry at a time.
struct GemmBatch {
  std::vector<const double*> X, Y, Z;
  std::vector<double*> D;
  void add(const double* x, const double* y, const double* z, double* d) {
    X.push_back(x);
    Y.push_back(y);
    Z.push_back(z);
    D.push_back(d);
  }
  int4 dense = make_int4(-1024, 1024, -1024, 1024);
  void flush(Schedule& s, double alpha, double beta) { flush(s, alpha, beta, dense); }
  void flush(Schedule& s, double alpha, double beta, int4 bp, int lane = 0) {
    s.gemm(alpha, beta, bp, X, Y, Z, D, lane);
    X.clear(); Y.clear(); Z.clear(); D.clear();
  }
};

struct InvBatch {
  std::vector<const double*> X;
  std::vector<double*> Y;
  void add(const double* x, double* y) {
    X.push_back(x);
    Y.push_back(y);
  }
  void flush(Schedule& s) {
    s.inv(X, Y);
    X.clear(); Y.clear();
  }
};

// Runs an uploaded schedule (pointer table dtab) of batched GEMMs and
// inverses on `st`; singular pivots set dstatus[0].  With gstatus non-null
// and M = 128, the dense products run on the tensor cores from BF16 digit
// slices (gemm_digits.cu: an FP64-level bound, FP64 issue rate left behind);
// a bounded wait that gives up there sets *gstatus.
bt_status run_schedule(const Schedule& sc, const double** dtab, int M, int* dstatus, cudaStream_t st,
                       int* gstatus = nullptr) {
  const size_t MM = (size_t)M * M;
  const int use_smem = M <= INV_SMEM_MAX ? 1 : 0;
  const size_t inv_smem = use_smem ? (MM + M) * sizeof(double) + M * sizeof(int)
                                   : M * sizeof(double) + M * sizeof(int);
  BT_CUDA(cudaFuncSetAttribute(k_inverse_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_smem));
  const int inv_threads = (int)std::min<size_t>(1024, std::max<size_t>(32, ((MM + 31) / 32) * 32));
  // Cluster inversion (M <= 256): C = 2, 4 or 8 CTAs per matrix.  Each launch
  // takes the largest C (at least 16 columns per CTA, its share of the matrix
  // in shared memory) whose clusters for the whole batch fit on the GPU at
  // once, else the smallest usable C; the one-CTA kernel when none is usable.
  struct CluCfg {
    int C = 0, threads = 0, fit = 0;  // fit: clusters resident at once
    size_t smem = 0;
  } clu[3];
  for (int ci = 0; ci < 3; ++ci) {
    const int C = 2 << ci, Mc = (M + C - 1) / C;
    CluCfg& cc = clu[ci];
    cc.smem = inv_cluster_smem(M, C);
    cc.threads = inv_cluster_threads(M, C);
    if (M < 32 || M > kInvClusterMaxM || (C > 2 && Mc < 16) || cc.smem > 200 * 1024) continue;
    if (cudaFuncSetAttribute(k_inverse_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cc.smem) !=
        cudaSuccess)
      continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(cc.threads);
    cfg.dynamicSmemBytes = cc.smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_inverse_cluster, &cfg) == cudaSuccess && n > 0) {
      cc.C = C;
      cc.fit = n;
    }
  }
  cudaGetLastError();
  const bool clu_ok = clu[0].C || clu[1].C || clu[2].C;
  size_t clu_attr = 0;  // the dynamic shared memory the kernel is currently set up for
  // GEMM tile: 32 when 64-tiles would pad the block by more than about 15 % in area
  const int pad64 = (M + 63) / 64 * 64, pad32 = (M + 31) / 32 * 32;
  // M <= 192: 16 x 16 tiles -- every launch holds 16x the CTAs of 64-tiles, which
  // evens out the waves over the SMs and shortens each CTA's FP64 chain
  // (measured at N=2048, M=128, S=64: 109 -> 86 ms per factorisation; M=64: 50 -> 32 ms)
  const int GT = M <= 192 ? 16 : ((double)pad32 * pad32 < 0.85 * (double)pad64 * pad64 ? 32 : 64);
  const int tiles = (M + GT - 1) / GT;
  // digit-slice products: scratch per lane (the lanes run concurrently)
  auto dense = [&](const Op& o) {
    return o.bp.x <= -(M - 1) && o.bp.y >= M - 1 && o.bp.z <= -(M - 1) && o.bp.w >= M - 1;
  };
  const bool dig = gstatus != nullptr && digit_gemm_supported(M);
  int emax = 0;
  bool lane1_dense = false;
  if (dig)
    for (const Op& o : sc.ops)
      if (o.kind == 0 && dense(o)) {
        emax = std::max(emax, std::min(o.batch, 65535));
        lane1_dense = lane1_dense || o.lane == 1;
      }
  void* dbuf[2] = {nullptr, nullptr};
  for (int l = 0; l < (lane1_dense ? 2 : 1) && emax > 0; ++l)
    BT_CUDA(cudaMallocAsync(&dbuf[l], digit_gemm_bytes(emax), st));
  // lane 1: created on first use, lowest priority (lane 0 holds the critical path)
  cudaStream_t lane1 = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool pending1 = false;  // lane 1 has work lane 0 has not joined
  for (const Op& o : sc.ops) {
    if (o.kind == 2) {
      if (pending1) {
        BT_CUDA(cudaEventRecord(ev1, lane1));
        BT_CUDA(cudaStreamWaitEvent(st, ev1, 0));
        pending1 = false;
      }
      continue;
    }
    cudaStream_t q = st;
    if (o.lane == 1) {
      if (!lane1) {
        int lo = 0, hi = 0;
        BT_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        BT_CUDA(cudaStreamCreateWithPriority(&lane1, cudaStreamNonBlocking, lo));
        BT_CUDA(cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming));
        BT_CUDA(cudaEventCreateWithFlags(&ev1, cudaEventDisableTiming));
      }
      BT_CUDA(cudaEventRecord(ev0, st));
      BT_CUDA(cudaStreamWaitEvent(lane1, ev0, 0));
      q = lane1;
      pending1 = true;
    }
    // grid.z / grid.x limits: split very large batches
    for (int b0 = 0; b0 < o.batch; b0 += 65535) {
      int nb = std::min(65535, o.batch - b0);
      if (o.kind == 3) {
        dim3 grid((unsigned)((MM + 1023) / 1024), (unsigned)nb);
        k_copy_blocks<<<grid, 256, 0, q>>>(dtab + o.off + 2 * (size_t)b0, MM);
      } else if (o.kind == 0 && emax > 0 && dense(o)) {
        BT_TRY(digit_gemm_run(dbuf[o.lane], emax, dtab + o.off + 4 * (size_t)b0, nb, o.alpha, o.beta, gstatus, q));
      } else if (o.kind == 0) {
        dim3 grid(tiles, tiles, nb);
        if (GT == 16)
          k_gemm_batched<16><<<grid, 256, 0, q>>>(dtab + o.off + 4 * (size_t)b0, M, o.alpha, o.beta, o.bp);
        else if (GT == 32)
          k_gemm_batched<32><<<grid, 256, 0, q>>>(dtab + o.off + 4 * (size_t)b0, M, o.alpha, o.beta, o.bp);
        else
          k_gemm_batched<64><<<grid, 256, 0, q>>>(dtab + o.off + 4 * (size_t)b0, M, o.alpha, o.beta, o.bp);
      } else {
        if (clu_ok) {
          int ci = -1;
          for (int c = 2; c >= 0 && ci < 0; --c)
            if (clu[c].C && nb <= clu[c].fit) ci = c;
          for (int c = 0; c < 3 && ci < 0; ++c)
            if (clu[c].C) ci = c;
          const CluCfg& cc = clu[ci];
          if (clu_attr < cc.smem) {
            BT_CUDA(cudaFuncSetAttribute(k_inverse_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cc.smem));
            clu_attr = cc.smem;
          }
          cudaLaunchConfig_t cfg = {};
          cfg.gridDim = dim3(cc.C * nb);
          cfg.blockDim = dim3(cc.threads);
          cfg.dynamicSmemBytes = cc.smem;
          cfg.stream = q;
          cudaLaunchAttribute at[1];
          at[0].id = cudaLaunchAttributeClusterDimension;
          at[0].val.clusterDim.x = cc.C;
          at[0].val.clusterDim.y = 1;
          at[0].val.clusterDim.z = 1;
          cfg.attrs = at;
          cfg.numAttrs = 1;
          BT_CUDA(cudaLaunchKernelEx(&cfg, k_inverse_cluster, dtab + o.off + 2 * (size_t)b0, M, dstatus));
        } else {
          k_inverse_batched<<<nb, inv_threads, inv_smem, q>>>(dtab + o.off + 2 * (size_t)b0, M, use_smem, dstatus);
        }
      }
    }
  }
  if (pending1) {
    BT_CUDA(cudaEventRecord(ev1, lane1));
    BT_CUDA(cudaStreamWaitEvent(st, ev1, 0));
  }
  for (void* b : dbuf)
    if (b) BT_CUDA(cudaFreeAsync(b, st));  // after lane 1's work (joined above)
  if (lane1) {
    // the stream and events may go once the work is enqueued (their
    // destruction is deferred until it completes)
    cudaStreamDestroy(lane1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
  }
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

}  // namespace

std::vector<TreeNode> build_tree(int S, int* depth_out) {
  std::vector<TreeNode> out;
  std::vector<TreeNode> cur{{0, S - 1, 0, 0}};
  int level = 0;
  while (!cur.empty()) {
    std::vector<TreeNode> next;
    for (auto n : cur) {
      if (n.l > n.r) continue;
      n.m = n.l + (n.r - n.l) / 2;
      n.level = level;
      out.push_back(n);
      if (n.l <= n.m - 1) next.push_back({n.l, n.m - 1, 0, level + 1});
      if (n.m + 1 <= n.r) next.push_back({n.m + 1, n.r, 0, level + 1});
    }
    cur.swap(next);
    ++level;
  }
  *depth_out = level;
  return out;
}

bt_status factor_f64(bt_handle_s* h, const double* A_in, const double* B_in, const double* C_in,
                     cudaStream_t st) {
  const int64_t N = h->N, S = h->S, L = h->L;
  const int M = (int)h->M;
  const size_t MM = (size_t)M * M;
  DevArena& ar = h->arena;

  // -- operator copies (A_1 and B_N zeroed) --------------------------------
  BT_TRY(ar.alloc((void**)&h->A, N * MM * sizeof(double)));
  BT_TRY(ar.alloc((void**)&h->B, N * MM * sizeof(double)));
  BT_TRY(ar.alloc((void**)&h->C, N * MM * sizeof(double)));
  k_copy<<<1024, 256, 0, st>>>(A_in, h->A, N * MM);
  k_copy<<<1024, 256, 0, st>>>(B_in, h->B, N * MM);
  k_copy<<<1024, 256, 0, st>>>(C_in, h->C, N * MM);
  BT_CUDA(cudaGetLastError());
  BT_CUDA(cudaMemsetAsync(h->A, 0, MM * sizeof(double), st));
  BT_CUDA(cudaMemsetAsync(h->B + (N - 1) * MM, 0, MM * sizeof(double), st));

  // -- diagonal bands of A_j and B_j (structure the GEMMs below skip) -------
  {
    int* dprof = nullptr;
    int hprof[4] = {INT_MAX, INT_MIN, INT_MAX, INT_MIN};
    BT_CUDA(cudaMallocAsync((void**)&dprof, sizeof(hprof), st));
    BT_CUDA(cudaMemcpyAsync(dprof, hprof, sizeof(hprof), cudaMemcpyHostToDevice, st));
    k_band_profile<<<1024, 256, 0, st>>>(h->A, h->B, N, M, dprof);
    BT_CUDA(cudaGetLastError());
    BT_CUDA(cudaMemcpyAsync(hprof, dprof, sizeof(hprof), cudaMemcpyDeviceToHost, st));
    BT_CUDA(cudaStreamSynchronize(st));
    BT_CUDA(cudaFreeAsync(dprof, st));
    // an all-zero operand lies in any band: take the main diagonal
    for (int k = 0; k < 4; k += 2)
      if (hprof[k] > hprof[k + 1]) hprof[k] = hprof[k + 1] = 0;
    for (int k = 0; k < 4; ++k) h->band[k] = hprof[k];
  }

  // -- factor arrays --------------------------------------------------------
  for (double** p : {&h->Dinv, &h->E, &h->G, &h->U, &h->V}) {
    BT_TRY(ar.alloc((void**)p, N * MM * sizeof(double)));
    BT_CUDA(cudaMemsetAsync(*p, 0, N * MM * sizeof(double), st));
  }
  for (double** p : {&h->At, &h->Ct, &h->Bt, &h->HL, &h->HR}) {
    BT_TRY(ar.alloc((void**)p, S * MM * sizeof(double)));
    BT_CUDA(cudaMemsetAsync(*p, 0, S * MM * sizeof(double), st));
  }
  int depth = 0;
  h->nodes = build_tree((int)S, &depth);
  h->depth = depth;
  BT_TRY(ar.alloc((void**)&h->R, (size_t)depth * S * MM * sizeof(double)));
  BT_CUDA(cudaMemsetAsync(h->R, 0, (size_t)depth * S * MM * sizeof(double), st));

  // work buffers: D / Sigma, T, invDL/invDR (per interface), identity, zero
  double *Dw, *Tw, *Iw, *Zw, *Pw;
  BT_TRY(ar.alloc((void**)&Dw, S * MM * sizeof(double)));
  BT_TRY(ar.alloc((void**)&Tw, S * MM * sizeof(double)));
  BT_TRY(ar.alloc((void**)&Pw, S * MM * sizeof(double)));
  BT_TRY(ar.alloc((void**)&Iw, MM * sizeof(double)));
  BT_TRY(ar.alloc((void**)&Zw, MM * sizeof(double)));
  k_set_identity<<<(int)((MM + 255) / 256), 256, 0, st>>>(Iw, M);
  BT_CUDA(cudaMemsetAsync(Zw, 0, MM * sizeof(double), st));

  auto blk = [&](double* base, int64_t j) { return base + (size_t)j * MM; };
  auto Aj = [&](int64_t j) -> const double* { return j == 0 ? Zw : blk(h->A, j); };
  auto Bj = [&](int64_t j) -> const double* { return j == N - 1 ? Zw : blk(h->B, j); };

  Schedule sc;
  sc.ident = Iw;
  GemmBatch g;
  InvBatch iv;
  // GEMM operand bands: A_j or B_j on the left (onX) or on the right (onY)
  const int4 dense = g.dense;
  auto onX = [&](int lo, int hi) { return make_int4(lo, hi, dense.z, dense.w); };
  auto onY = [&](int lo, int hi) { return make_int4(dense.x, dense.y, lo, hi); };
  const int4 xA = onX(h->band[0], h->band[1]), xB = onX(h->band[2], h->band[3]);
  const int4 yA = onY(h->band[0], h->band[1]), yB = onY(h->band[2], h->band[3]);
  // one batch for A and B operands together when their bands coincide
  const bool split = h->band[0] != h->band[2] || h->band[1] != h->band[3];

  // ---- step 1.1: block sweep factorisation of every segment interior ------
  // The forward products of E of eq. sub1 (Y_i = E_i Y_{i-1}, kept in U until
  // the backward products) trail the sweep by one row on lane 1: row t-1's
  // product runs beside row t's pivot inversions, which hold only S SMs.
  auto y_step = [&](int64_t t) {
    for (int64_t s = 0; s < S; ++s) {
      int64_t i = s * L + t;
      g.add(blk(h->E, i), t == 1 ? Iw : blk(h->U, i - 1), nullptr, blk(h->U, i));
    }
    g.flush(sc, 1.0, 0.0, g.dense, 1);
  };
  for (int64_t t = 1; t < L; ++t) {
    if (t > 1) {
      for (int64_t s = 0; s < S; ++s) {
        int64_t i = s * L + t;
        g.add(Aj(i), blk(h->G, i - 1), blk(h->C, i), blk(Dw, s));
      }
      g.flush(sc, -1.0, 1.0, xA);  // D = C_i - A_i G_{i-1}
      y_step(t - 1);
      for (int64_t s = 0; s < S; ++s) iv.add(blk(Dw, s), blk(h->Dinv, s * L + t));
    } else {
      for (int64_t s = 0; s < S; ++s) iv.add(blk(h->C, s * L + t), blk(h->Dinv, s * L + t));
    }
    iv.flush(sc);
    for (int64_t s = 0; s < S; ++s) g.add(blk(h->Dinv, s * L + t), Bj(s * L + t), nullptr, blk(h->G, s * L + t));
    if (split) g.flush(sc, 1.0, 0.0, yB);
    for (int64_t s = 0; s < S; ++s) g.add(blk(h->Dinv, s * L + t), Aj(s * L + t), nullptr, blk(h->E, s * L + t));
    g.flush(sc, 1.0, 0.0, yA);
  }
  // V (eq. sub2): backward products of G
  for (int64_t t = L - 1; t >= 1; --t) {
    for (int64_t s = 0; s < S; ++s) {
      int64_t i = s * L + t;
      g.add(blk(h->G, i), t == L - 1 ? Iw : blk(h->V, i + 1), nullptr, blk(h->V, i));
    }
    g.flush(sc, 1.0, 0.0);
  }
  // U (eq. sub1): the last forward product, then U_i = Y_i + G_i U_{i+1}
  if (L > 1) y_step(L - 1);
  sc.join();
  for (int64_t t = L - 2; t >= 1; --t) {
    for (int64_t s = 0; s < S; ++s) {
      int64_t i = s * L + t;
      g.add(blk(h->G, i), blk(h->U, i + 1), blk(h->U, i), blk(h->U, i));
    }
    g.flush(sc, 1.0, 1.0);
  }

  // ---- step 1.2: reduced system of eq. red1 -------------------------------
  // Neighbour responses: rows K-1 / K+1 in the representation of segments
  // s-1 / s; with L = 1 those rows are interfaces (U = I, V = 0 on the left;
  // U = 0, V = I on the right).
  auto Ul = [&](int64_t s) -> const double* { return s == 0 ? Zw : (L == 1 ? Iw : blk(h->U, s * L - 1)); };
  auto Vl = [&](int64_t s) -> const double* { return s == 0 ? Zw : (L == 1 ? Zw : blk(h->V, s * L - 1)); };
  auto Ur = [&](int64_t s) -> const double* { return s * L + 1 >= N ? Zw : (L == 1 ? Zw : blk(h->U, s * L + 1)); };
  auto Vr = [&](int64_t s) -> const double* { return s * L + 1 >= N ? Zw : (L == 1 ? Iw : blk(h->V, s * L + 1)); };
  for (int64_t s = 0; s < S; ++s) g.add(Aj(s * L), Ul(s), nullptr, blk(h->At, s));
  if (split) g.flush(sc, 1.0, 0.0, xA);
  for (int64_t s = 0; s < S; ++s) g.add(Bj(s * L), Vr(s), nullptr, blk(h->Bt, s));
  g.flush(sc, 1.0, 0.0, xB);
  for (int64_t s = 0; s < S; ++s) g.add(Aj(s * L), Vl(s), blk(h->C, s * L), blk(h->Ct, s));
  g.flush(sc, -1.0, 1.0, xA);
  for (int64_t s = 0; s < S; ++s) g.add(Bj(s * L), Ur(s), blk(h->Ct, s), blk(h->Ct, s));
  g.flush(sc, -1.0, 1.0, xB);

  // ---- step 1.3: rows of the inverses for Algorithm 1 on P~ ---------------
  // The Schur-complement chains of a node and the propagation of its block
  // row depend only on the reduced system, so the levels are independent:
  // with work buffers per level (Pw: DL_j^{-1} / DR_j^{-1}, Dw: DL_j / DR_j /
  // Sigma, Tw: products) the chains of ALL levels advance together, t steps
  // for the longest chain instead of the sum over levels, in batches that
  // hold every level's blocks.  Past a memory budget the levels run one
  // after the other on shared buffers.
  h->level_off.assign(depth + 1, 0);
  for (auto& n : h->nodes) h->level_off[n.level + 1]++;
  for (int l = 0; l < depth; ++l) h->level_off[l + 1] += h->level_off[l];
  auto Rb = [&](int level, int j) { return h->R + ((size_t)level * S + j) * MM; };
  const bool together = depth > 1 && 3.0 * depth * S * MM * sizeof(double) <= 4.0 * (1ull << 30);
  double *PwL = Pw, *DwL = Dw, *TwL = Tw;
  double* lvl_buf = nullptr;  // released once the schedule has run
  if (together) {
    const size_t lvl = (size_t)depth * S * MM;
    if (cudaMallocAsync((void**)&lvl_buf, 3 * lvl * sizeof(double), st) != cudaSuccess) {
      cudaGetLastError();
      set_error("bt_factor: work buffer allocation failed");
      return BT_ERR_OOM;
    }
    PwL = lvl_buf;
    DwL = lvl_buf + lvl;
    TwL = lvl_buf + 2 * lvl;
  }
  auto lb = [&](double* base, int lev, int j) { return base + ((size_t)(together ? lev : 0) * S + j) * MM; };
  for (int g0 = 0; g0 < depth; g0 = together ? depth : g0 + 1) {
    const int g1 = together ? depth : g0 + 1;
    struct LN {
      TreeNode n;
      int lev;
    };
    std::vector<LN> ns;
    for (int lev = g0; lev < g1; ++lev)
      for (int q = h->level_off[lev]; q < h->level_off[lev + 1]; ++q) ns.push_back({h->nodes[q], lev});
    int maxlen = 0;
    for (auto& x : ns) maxlen = std::max(maxlen, std::max(x.n.m - x.n.l, x.n.r - x.n.m));
    // chains of Schur complements from both ends towards m
    for (int t = 0; t < maxlen; ++t) {
      bool any = false;
      for (auto& x : ns) {
        const TreeNode& n = x.n;
        if (t > 0 && t < n.m - n.l) {
          int j = n.l + t;
          g.add(blk(h->At, j), lb(PwL, x.lev, j - 1), nullptr, lb(TwL, x.lev, j));
          any = true;
        }
        if (t > 0 && t < n.r - n.m) {
          int j = n.r - t;
          g.add(blk(h->Bt, j), lb(PwL, x.lev, j + 1), nullptr, lb(TwL, x.lev, j));
          any = true;
        }
      }
      if (any) g.flush(sc, 1.0, 0.0);
      for (auto& x : ns) {
        const TreeNode& n = x.n;
        if (t > 0 && t < n.m - n.l) {
          int j = n.l + t;
          g.add(lb(TwL, x.lev, j), blk(h->Bt, j - 1), blk(h->Ct, j), lb(DwL, x.lev, j));
        }
        if (t > 0 && t < n.r - n.m) {
          int j = n.r - t;
          g.add(lb(TwL, x.lev, j), blk(h->At, j + 1), blk(h->Ct, j), lb(DwL, x.lev, j));
        }
      }
      g.flush(sc, -1.0, 1.0);
      for (auto& x : ns) {
        const TreeNode& n = x.n;
        if (t < n.m - n.l) {
          int j = n.l + t;
          iv.add(t == 0 ? blk(h->Ct, j) : lb(DwL, x.lev, j), lb(PwL, x.lev, j));
        }
        if (t < n.r - n.m) {
          int j = n.r - t;
          iv.add(t == 0 ? blk(h->Ct, j) : lb(DwL, x.lev, j), lb(PwL, x.lev, j));
        }
      }
      iv.flush(sc);
    }
    // Sigma_m and R_mm
    for (auto& x : ns) {
      const TreeNode& n = x.n;
      g.add(n.m > n.l ? blk(h->At, n.m) : Zw, n.m > n.l ? lb(PwL, x.lev, n.m - 1) : Zw, nullptr,
            lb(TwL, x.lev, n.m));
    }
    g.flush(sc, 1.0, 0.0);
    for (auto& x : ns) {
      const TreeNode& n = x.n;
      g.add(lb(TwL, x.lev, n.m), n.m > n.l ? blk(h->Bt, n.m - 1) : Zw, blk(h->Ct, n.m), lb(DwL, x.lev, n.m));
    }
    g.flush(sc, -1.0, 1.0);
    for (auto& x : ns) {
      const TreeNode& n = x.n;
      g.add(n.m < n.r ? blk(h->Bt, n.m) : Zw, n.m < n.r ? lb(PwL, x.lev, n.m + 1) : Zw, nullptr,
            lb(TwL, x.lev, n.m));
    }
    g.flush(sc, 1.0, 0.0);
    for (auto& x : ns) {
      const TreeNode& n = x.n;
      g.add(lb(TwL, x.lev, n.m), n.m < n.r ? blk(h->At, n.m + 1) : Zw, lb(DwL, x.lev, n.m), lb(DwL, x.lev, n.m));
    }
    g.flush(sc, -1.0, 1.0);
    for (auto& x : ns) iv.add(lb(DwL, x.lev, x.n.m), Rb(x.lev, x.n.m));
    iv.flush(sc);
    // propagate the block row outwards
    for (int t = 1; t <= maxlen; ++t) {
      for (auto& x : ns) {
        const TreeNode& n = x.n;
        if (t <= n.m - n.l) {
          int j = n.m - t;
          g.add(Rb(x.lev, j + 1), blk(h->At, j + 1), nullptr, lb(TwL, x.lev, j));
        }
        if (t <= n.r - n.m) {
          int j = n.m + t;
          g.add(Rb(x.lev, j - 1), blk(h->Bt, j - 1), nullptr, lb(TwL, x.lev, j));
        }
      }
      g.flush(sc, 1.0, 0.0);
      for (auto& x : ns) {
        const TreeNode& n = x.n;
        if (t <= n.m - n.l) {
          int j = n.m - t;
          g.add(lb(TwL, x.lev, j), lb(PwL, x.lev, j), nullptr, Rb(x.lev, j));
        }
        if (t <= n.r - n.m) {
          int j = n.m + t;
          g.add(lb(TwL, x.lev, j), lb(PwL, x.lev, j), nullptr, Rb(x.lev, j));
        }
      }
      g.flush(sc, 1.0, 0.0);
    }
    for (auto& x : ns) {
      const TreeNode& n = x.n;
      if (n.l > 0) g.add(Rb(x.lev, n.l), blk(h->At, n.l), nullptr, blk(h->HL, n.m));
      if (n.r < S - 1) g.add(Rb(x.lev, n.r), blk(h->Bt, n.r), nullptr, blk(h->HR, n.m));
    }
    g.flush(sc, 1.0, 0.0);
  }

  // ---- upload the schedule and run it --------------------------------------
  const double** dtab = nullptr;
  int* dstatus = nullptr;
  BT_CUDA(cudaMallocAsync((void**)&dtab, std::max<size_t>(1, sc.tab.size()) * sizeof(double*), st));
  BT_CUDA(cudaMallocAsync((void**)&dstatus, 4 * sizeof(int), st));
  BT_CUDA(cudaMemsetAsync(dstatus, 0, 4 * sizeof(int), st));
  BT_CUDA(cudaMemcpyAsync(dtab, sc.tab.data(), sc.tab.size() * sizeof(double*), cudaMemcpyHostToDevice, st));

  BT_TRY(run_schedule(sc, dtab, M, dstatus, st, dstatus + 3));

  // stencil detection (A_j = B_j = I, tridiagonal C_j) for the residual
  k_detect_stencil<<<1024, 256, 0, st>>>(h->A, h->B, h->C, N, M, dstatus + 1);
  BT_CUDA(cudaGetLastError());
  // interface coupling blocks and the tridiagonal part of C
  BT_TRY(ar.alloc((void**)&h->AK, S * MM * sizeof(double)));
  BT_TRY(ar.alloc((void**)&h->BK, S * MM * sizeof(double)));
  BT_TRY(ar.alloc((void**)&h->Cdiag, (size_t)N * M * 3 * sizeof(double)));
  BT_TRY(ar.alloc((void**)&h->Cdw, (size_t)N * M * 2 * sizeof(float)));
  k_gather_blocks<<<256, 256, 0, st>>>(h->A, h->AK, S, L, MM);
  k_gather_blocks<<<256, 256, 0, st>>>(h->B, h->BK, S, L, MM);
  k_tridiag<<<256, 256, 0, st>>>(h->C, h->Cdiag, h->Cdw, N, M, dstatus + 2);
  BT_CUDA(cudaGetLastError());

  // tree tables for the solve kernels
  std::vector<int> hn(3 * h->nodes.size()), hml(S, 0);
  for (size_t q = 0; q < h->nodes.size(); ++q) {
    hn[3 * q] = h->nodes[q].l;
    hn[3 * q + 1] = h->nodes[q].r;
    hn[3 * q + 2] = h->nodes[q].m;
    hml[h->nodes[q].m] = h->nodes[q].level;
  }
  BT_TRY(ar.alloc((void**)&h->d_nodes, hn.size() * sizeof(int)));
  BT_TRY(ar.alloc((void**)&h->d_mid_level, S * sizeof(int)));
  BT_CUDA(cudaMemcpyAsync(h->d_nodes, hn.data(), hn.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  BT_CUDA(cudaMemcpyAsync(h->d_mid_level, hml.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));

  int hstatus[4] = {0, 0, 0, 0};
  BT_CUDA(cudaMemcpyAsync(hstatus, dstatus, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  BT_CUDA(cudaStreamSynchronize(st));
  BT_CUDA(cudaFreeAsync(dtab, st));
  BT_CUDA(cudaFreeAsync(dstatus, st));
  if (lvl_buf) BT_CUDA(cudaFreeAsync(lvl_buf, st));
  h->stencil = hstatus[1] ? 0 : 1;
  h->stencil_unit = (h->stencil && !hstatus[2]) ? 1 : 0;
  if (hstatus[3]) {
    set_error("bt_factor: a bounded wait of the tensor-core block products gave up");
    return BT_ERR_TIMEOUT;
  }
  if (hstatus[0]) {
    set_error("bt_factor: a pivot block of the block sweep or of the reduced system is singular or non-finite");
    return BT_ERR_SINGULAR;
  }
  return BT_OK;
}

// The forward responses of the left interface coupling, Y_a = E_a and
// Y_i = E_i Y_{i-1} on the interior rows a..b of every segment (the part of
// eq. sub1 before the backward products), into h->Y ([N][M][M] FP64,
// interface rows zero); built on first use by the tensor-core stage 2 of
// unit stencils, whose backward pass applies Y_i X~_s row by row.
bt_status factor_left_responses(bt_handle_s* h, cudaStream_t st) {
  if (h->Y) return BT_OK;
  const int64_t N = h->N, S = h->S, L = h->L;
  const int M = (int)h->M;
  const size_t MM = (size_t)M * M;
  double* Y = nullptr;
  BT_TRY(h->arena.alloc((void**)&Y, N * MM * sizeof(double)));
  BT_CUDA(cudaMemsetAsync(Y, 0, N * MM * sizeof(double), st));
  double* Iw = nullptr;
  BT_CUDA(cudaMallocAsync((void**)&Iw, MM * sizeof(double), st));
  k_set_identity<<<(int)((MM + 255) / 256), 256, 0, st>>>(Iw, M);
  BT_CUDA(cudaGetLastError());
  Schedule sc;
  sc.ident = Iw;
  GemmBatch g;
  auto blk = [&](double* base, int64_t j) { return base + (size_t)j * MM; };
  for (int64_t t = 1; t < L; ++t) {
    for (int64_t s = 0; s < S; ++s) {
      const int64_t i = s * L + t;
      g.add(blk(h->E, i), t == 1 ? Iw : blk(Y, i - 1), nullptr, blk(Y, i));
    }
    g.flush(sc, 1.0, 0.0);
  }
  const double** dtab = nullptr;
  int* dstatus = nullptr;
  BT_CUDA(cudaMallocAsync((void**)&dtab, std::max<size_t>(1, sc.tab.size()) * sizeof(double*), st));
  BT_CUDA(cudaMallocAsync((void**)&dstatus, sizeof(int), st));
  BT_CUDA(cudaMemsetAsync(dstatus, 0, sizeof(int), st));
  BT_CUDA(cudaMemcpyAsync(dtab, sc.tab.data(), sc.tab.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
  BT_TRY(run_schedule(sc, dtab, M, dstatus, st));
  BT_CUDA(cudaStreamSynchronize(st));  // the host table goes out of scope
  BT_CUDA(cudaFreeAsync(dtab, st));
  BT_CUDA(cudaFreeAsync(dstatus, st));
  BT_CUDA(cudaFreeAsync(Iw, st));
  h->Y = Y;
  return BT_OK;
}

}  // namespace bt
