// Schur-complement CG with a probing band preconditioner (Section 3.3, eqs.
// schur_decomp and domains_equation; Section 3.3.2 for the probing).
//
// Model problem: the five-point operator (4 + shift) x - (four neighbours) on
// an nz x nr grid, cut by p - 1 interface grid rows into p strips of h rows
// (nz = p h + p - 1; strip i = rows i (h + 1) .. + h - 1; line k = row
// k (h + 1) + h).  Every strip operator, its unknowns ordered by grid column,
// is block tridiagonal (N = nr blocks of M = h: A_j = B_j = I, C_j =
// tridiag(-1, 4 + shift, -1)); all p strips share it, so one factorisation
// serves them and the p strips of one product are solved together as p K
// right-hand-side columns of one dichotomy solve.
//
//   product with S:   w = A_II^{-1} (E v),  (S v)_k = A_GG v_k - w_k[h-1] - w_{k+1}[0]
//   right-hand side:  u = A_II^{-1} f_I,    g_k = f_G,k + u_k[h-1] + u_{k+1}[0]
//   recovery:         x_I = A_II^{-1} (f_I + E x_G)
// where E v puts line k's values on the last row of strip k and the first row
// of strip k + 1 (A_IG = -E, A_GI = -E^T), and A_GG = tridiag(-1, 4 + shift, -1)
// along a line.
//
// Probing: the 2d+1 vectors p_l (1 where the interface index is l mod 2d+1)
// go through one product with S (K = 2d+1); B[i][j] = (S p_{j mod w})[i] for
// |i - j| <= d, symmetrised, in diagonal-ordered band storage, factored by
// bt_factor_band.  d = -1: no preconditioner.
//
// PCG (Saad, Algorithm 9.1) runs for all K columns at once; a column stops
// once ||r|| <= tol ||g|| (its step length is zero from then on).  Column dot
// products are deterministic (fixed reduction order); the host reads one
// count of active columns per iteration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "bt_internal.cuh"

struct bt_schur_s {
  int device = 0;
  int64_t nr = 0, h = 0, p = 0, nz = 0, ng = 0, d = -1, S = 1, MB = 0, SB = 0;
  double shift = 0.0;
  bt_handle strip = nullptr;  // factored strip operator
  bt_handle band = nullptr;   // factored preconditioner B (d >= 0)
  double* ab = nullptr;       // B in band storage [2d+1][ng]
  double* sbuf = nullptr;     // strip panels Fs, Ws: [nr][h][p K] each
  size_t sbytes = 0;
  double* vbuf = nullptr;     // interface panels g, x, r, z, pd, q: [ng][K] each
  size_t vbytes = 0;
  double* cbuf = nullptr;     // per-column scalars: rz, rz', pq, rr, gn2
  int* ibuf = nullptr;        // active flags [K] + active count + iteration count
  size_t cK = 0;
  // The PCG solve as one CUDA graph (prologue, device-side WHILE over the
  // iterations, epilogue) for the last argument key; `ptrs` are the buffers
  // it was captured with (a reallocation anywhere captures again).
  cudaGraphExec_t pcg_exec = nullptr;
  const double* pcg_F = nullptr;
  double* pcg_X = nullptr;
  int64_t pcg_K = 0;
  double pcg_tol = 0.0;
  int32_t pcg_max = -1;
  std::vector<const void*> pcg_ptrs;
  cudaStream_t cap = nullptr, cap2 = nullptr;
};

namespace bt {

namespace {

__global__ void k_strip_blocks(int64_t nr, int h, double diag, double* A, double* B, double* C) {
  const size_t hh = (size_t)h * h, tot = (size_t)nr * hh;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t j = (int64_t)(e / hh);
    const int r = (int)((e % hh) / h), c = (int)(e % h);
    A[e] = (j > 0 && r == c) ? 1.0 : 0.0;
    B[e] = (j < nr - 1 && r == c) ? 1.0 : 0.0;
    C[e] = r == c ? diag : ((r == c + 1 || c == r + 1) ? -1.0 : 0.0);
  }
}

// Fs[r][m][i K + c] = F[z(i, m)][r][c] (if F) + (E v) on the strip rows next
// to the interface lines (if v).
__global__ void k_strip_rhs(const double* __restrict__ F, const double* __restrict__ v, int64_t nr, int h, int p,
                            int64_t K, double* __restrict__ Fs) {
  const int64_t pK = (int64_t)p * K;
  const size_t tot = (size_t)nr * h * pK;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t col = (int64_t)(e % pK);
    const int64_t rm = (int64_t)(e / pK);
    const int m = (int)(rm % h);
    const int64_t r = rm / h;
    const int i = (int)(col / K);
    const int64_t c = col % K;
    double s = 0.0;
    if (F) s = F[((int64_t)(i * (h + 1) + m) * nr + r) * K + c];
    if (v) {
      if (m == 0 && i > 0) s += v[((int64_t)(i - 1) * nr + r) * K + c];
      if (m == h - 1 && i < p - 1) s += v[((int64_t)i * nr + r) * K + c];
    }
    Fs[e] = s;
  }
}

// mode 0: out = S v = A_GG v - w_k[h-1] - w_{k+1}[0];  mode 1: out = g = f_G + w_k[h-1] + w_{k+1}[0]
__global__ void k_iface_out(const double* __restrict__ v, const double* __restrict__ F,
                            const double* __restrict__ Ws, int64_t nr, int h, int p, int64_t K, double diag, int mode,
                            double* __restrict__ out) {
  const int64_t pK = (int64_t)p * K;
  const size_t tot = (size_t)(p - 1) * nr * K;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t c = (int64_t)(e % K);
    const int64_t kr = (int64_t)(e / K);
    const int64_t r = kr % nr;
    const int k = (int)(kr / nr);
    const double w = Ws[(r * h + (h - 1)) * pK + (int64_t)k * K + c] + Ws[(r * h) * pK + (int64_t)(k + 1) * K + c];
    if (mode == 0) {
      double s = diag * v[e];
      if (r > 0) s -= v[e - K];
      if (r < nr - 1) s -= v[e + K];
      out[e] = s - w;
    } else {
      out[e] = F[((int64_t)(k * (h + 1) + h) * nr + r) * K + c] + w;
    }
  }
}

// X[z][r][c]: interface rows from xg, strip rows from Ws
__global__ void k_grid_out(const double* __restrict__ Ws, const double* __restrict__ xg, int64_t nr, int h, int p,
                           int64_t K, double* __restrict__ X) {
  const int64_t pK = (int64_t)p * K;
  const int64_t nz = (int64_t)p * h + p - 1;
  const size_t tot = (size_t)nz * nr * K;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t c = (int64_t)(e % K);
    const int64_t zr = (int64_t)(e / K);
    const int64_t r = zr % nr;
    const int64_t z = zr / nr;
    const int i = (int)(z / (h + 1)), m = (int)(z % (h + 1));
    X[e] = m == h ? xg[((int64_t)i * nr + r) * K + c] : Ws[(r * h + m) * pK + (int64_t)i * K + c];
  }
}

__global__ void k_probe_vectors(int64_t ng, int w, double* P) {
  const size_t tot = (size_t)ng * w;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x)
    P[e] = ((int64_t)(e / w) % w == (int64_t)(e % w)) ? 1.0 : 0.0;
}

// ab[d + i - j][j] = (SP[i][j mod w] + SP[j][i mod w]) / 2 for |i - j| <= d
__global__ void k_probe_band(const double* __restrict__ SP, int64_t ng, int d, double* __restrict__ ab) {
  const int w = 2 * d + 1;
  const size_t tot = (size_t)w * ng;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t j = (int64_t)(e % ng);
    const int64_t i = (int64_t)(e / ng) - d + j;
    ab[e] = (i >= 0 && i < ng) ? 0.5 * (SP[i * w + j % w] + SP[j * w + i % w]) : 0.0;
  }
}

// out[c] = sum_i a[i][c] b[i][c], n rows, K columns; one 1024-thread block per
// 32 columns (fewer columns: several row lanes per column); fixed order.
__global__ void __launch_bounds__(1024) k_coldot(const double* __restrict__ a, const double* __restrict__ b,
                                                 int64_t n, int64_t K, double* __restrict__ out) {
  __shared__ double part[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  const int kc = K - c0 < 32 ? (int)(K - c0) : 32;
  const int lanes = 32 / kc;  // row lanes per column within a warp
  const int tx = threadIdx.x, ty = threadIdx.y;
  double s = 0.0;
  if (tx < kc * lanes) {
    const int64_t c = c0 + tx % kc;
    const int64_t step = 32 * (int64_t)lanes;
#pragma unroll 4
    for (int64_t i = (int64_t)ty * lanes + tx / kc; i < n; i += step) s = fma(a[i * K + c], b[i * K + c], s);
  }
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && tx < kc) {
    double t = 0.0;
    for (int y = 0; y < 32; ++y)
      for (int l = 0; l < lanes; ++l) t += part[y][l * kc + tx];
    out[c0 + tx] = t;
  }
}

// CG start: rz = +inf (so the first step takes beta = 0), every column active,
// no iteration yet
__global__ void k_pcg_init(double* rz, int64_t K, int* active, int* it) {
  for (int64_t c = threadIdx.x; c < K; c += blockDim.x) {
    rz[c] = INFINITY;
    active[c] = 1;
  }
  if (threadIdx.x == 0) *it = 0;
}

__global__ void k_copy_cols(double* __restrict__ dst, const double* __restrict__ src, int64_t K) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < K; c += (int64_t)gridDim.x * blockDim.x)
    dst[c] = src[c];
}

// active[c] &= rr[c] > tol^2 gn2[c]; count the active columns.  step 1 (after
// an iteration) also counts the iteration; the loop condition is set to
// "active columns remain and fewer than max_it iterations ran".
__global__ void k_pcg_check(const double* rr, const double* gn2, double tol2, int64_t K, int* active, int* count,
                            int* it, int max_it, int step, cudaGraphConditionalHandle loop) {
  int n = 0;
  for (int64_t c = threadIdx.x; c < K; c += blockDim.x) {
    const int a = active[c] && rr[c] > tol2 * gn2[c];
    active[c] = a;
    n += a;
  }
  n = __reduce_add_sync(0xffffffffu, n);
  __shared__ int wsum[32];
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
    *count = t;
    const int done = *it + step;
    *it = done;
    if (loop) cudaGraphSetConditional(loop, (t > 0 && done < max_it) ? 1u : 0u);
  }
}

__global__ void k_pcg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ pd,
                         const double* __restrict__ q, const double* __restrict__ rz, const double* __restrict__ pq,
                         const int* __restrict__ active, int64_t n, int64_t K) {
  const size_t tot = (size_t)n * K;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t c = (int64_t)(e % K);
    if (!active[c]) continue;
    const double alpha = rz[c] / pq[c];
    x[e] = fma(alpha, pd[e], x[e]);
    r[e] = fma(-alpha, q[e], r[e]);
  }
}

__global__ void k_pcg_p(double* __restrict__ pd, const double* __restrict__ z, const double* __restrict__ rz_new,
                        const double* __restrict__ rz, const int* __restrict__ active, int64_t n, int64_t K) {
  const size_t tot = (size_t)n * K;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t c = (int64_t)(e % K);
    const double beta = active[c] ? rz_new[c] / rz[c] : 0.0;
    pd[e] = fma(beta, pd[e], z[e]);
  }
}

// [a, a + na) and [b, b + nb) (doubles) share an element
bool overlap(const double* a, const double* b, size_t na, size_t nb = 0) {
  if (nb == 0) nb = na;
  return a < b + nb && b < a + na;
}

int grid_for(const void* fn, size_t tot) {
  return (int)std::max<size_t>(1, std::min<size_t>((tot + 255) / 256, (size_t)resident_grid(fn, 256, 0)));
}

#define EW(kern, tot, ...)                                                        \
  do {                                                                            \
    kern<<<grid_for((const void*)kern, (tot)), 256, 0, st>>>(__VA_ARGS__);        \
    BT_CUDA(cudaGetLastError());                                                  \
  } while (0)

bt_status coldot(const double* a, const double* b, int64_t n, int64_t K, double* out, cudaStream_t st) {
  k_coldot<<<(unsigned)((K + 31) / 32), dim3(32, 32), 0, st>>>(a, b, n, K, out);
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

bt_status grow(double** p, size_t* have, size_t need) {
  if (need <= *have) return BT_OK;
  BT_CUDA(cudaDeviceSynchronize());
  if (*p) BT_CUDA(cudaFree(*p));
  *p = nullptr;
  *have = 0;
  const cudaError_t e = cudaMalloc((void**)p, need);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error(std::string("schur: device allocation failed: ") + cudaGetErrorString(e));
    return BT_ERR_OOM;
  }
  *have = need;
  return BT_OK;
}

bt_status ensure_k(bt_schur_s* s, int64_t K) {
  BT_TRY(grow(&s->sbuf, &s->sbytes, 2 * (size_t)s->nr * s->h * s->p * K * sizeof(double)));
  BT_TRY(grow(&s->vbuf, &s->vbytes, 6 * (size_t)s->ng * K * sizeof(double)));
  if ((size_t)K > s->cK) {
    BT_CUDA(cudaDeviceSynchronize());
    if (s->cbuf) BT_CUDA(cudaFree(s->cbuf));
    if (s->ibuf) BT_CUDA(cudaFree(s->ibuf));
    s->cbuf = nullptr;
    s->ibuf = nullptr;
    s->cK = 0;
    BT_CUDA(cudaMalloc((void**)&s->cbuf, 5 * (size_t)K * sizeof(double)));
    BT_CUDA(cudaMalloc((void**)&s->ibuf, ((size_t)K + 2) * sizeof(int)));
    s->cK = (size_t)K;
  }
  return BT_OK;
}

// w = A_II^{-1} (F_I + E v) into the second strip panel (F or v may be null)
bt_status strip_solve(bt_schur_s* s, const double* F, const double* v, int64_t K, cudaStream_t st) {
  double* Fs = s->sbuf;
  double* Ws = s->sbuf + (size_t)s->nr * s->h * s->p * K;
  EW(k_strip_rhs, (size_t)s->nr * s->h * s->p * K, F, v, s->nr, (int)s->h, (int)s->p, K, Fs);
  return bt_solve(s->strip, Fs, s->p * K, Ws, st);
}

const double* strip_out(bt_schur_s* s, int64_t K) { return s->sbuf + (size_t)s->nr * s->h * s->p * K; }

bt_status apply_S(bt_schur_s* s, const double* v, int64_t K, double* out, cudaStream_t st) {
  BT_TRY(strip_solve(s, nullptr, v, K, st));
  EW(k_iface_out, (size_t)s->ng * K, v, nullptr, strip_out(s, K), s->nr, (int)s->h, (int)s->p, K, 4.0 + s->shift, 0,
     out);
  return BT_OK;
}

bt_status reduce_rhs(bt_schur_s* s, const double* F, int64_t K, double* g, cudaStream_t st) {
  BT_TRY(strip_solve(s, F, nullptr, K, st));
  EW(k_iface_out, (size_t)s->ng * K, nullptr, F, strip_out(s, K), s->nr, (int)s->h, (int)s->p, K, 4.0 + s->shift, 1,
     g);
  return BT_OK;
}

bt_status precond(bt_schur_s* s, const double* r, int64_t K, double* z, cudaStream_t st) {
  if (!s->band) {
    BT_CUDA(cudaMemcpyAsync(z, r, (size_t)s->ng * K * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return BT_OK;
  }
  bt_opts o;
  std::memset(&o, 0, sizeof(o));
  o.stream = st;
  return bt_solve_band(s->band, r, K, z, &o, nullptr);
}

void destroy(bt_schur_s* s) {
  if (!s) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  if (s->pcg_exec) cudaGraphExecDestroy(s->pcg_exec);
  if (s->cap) cudaStreamDestroy(s->cap);
  if (s->cap2) cudaStreamDestroy(s->cap2);
  if (s->strip) bt_destroy(s->strip);
  if (s->band) bt_destroy(s->band);
  for (void* q : {(void*)s->ab, (void*)s->sbuf, (void*)s->vbuf, (void*)s->cbuf, (void*)s->ibuf})
    if (q) cudaFree(q);
  cudaSetDevice(prev);
  delete s;
}

bt_status build(bt_schur_s* s, cudaStream_t st) {
  // strip operator, factored once for all strips
  const size_t hh = (size_t)s->h * s->h;
  double* blk = nullptr;
  BT_CUDA(cudaMallocAsync((void**)&blk, 3 * (size_t)s->nr * hh * sizeof(double), st));
  double *A = blk, *B = blk + (size_t)s->nr * hh, *C = blk + 2 * (size_t)s->nr * hh;
  k_strip_blocks<<<grid_for((const void*)k_strip_blocks, (size_t)s->nr * hh), 256, 0, st>>>(s->nr, (int)s->h,
                                                                                           4.0 + s->shift, A, B, C);
  bt_status rc = cudaGetLastError() == cudaSuccess ? BT_OK : BT_ERR_CUDA;
  if (rc == BT_OK) rc = bt_factor(s->nr, s->h, A, B, C, s->S, st, &s->strip);
  const cudaError_t fe = cudaFreeAsync(blk, st);
  if (rc != BT_OK) return rc;
  if (fe != cudaSuccess) return cuda_fail(fe, "cudaFreeAsync");
  if (s->d < 0) return BT_OK;
  // probing: S P with the 2d+1 probing vectors, band read-off, factorisation of B
  const int w = (int)(2 * s->d + 1);
  BT_TRY(ensure_k(s, w));
  double* P = s->vbuf;                       // [ng][w]
  double* SP = s->vbuf + (size_t)s->ng * w;  // [ng][w]
  EW(k_probe_vectors, (size_t)s->ng * w, s->ng, w, P);
  BT_TRY(apply_S(s, P, w, SP, st));
  BT_CUDA(cudaMalloc((void**)&s->ab, (size_t)w * s->ng * sizeof(double)));
  EW(k_probe_band, (size_t)w * s->ng, SP, s->ng, (int)s->d, s->ab);
  return bt_factor_band(s->ng, s->d, s->d, s->ab, s->MB, s->SB, st, &s->band);
}

}  // namespace
}  // namespace bt

using namespace bt;

extern "C" {

bt_status bt_schur_create(int64_t nr, int64_t h, int64_t p, double shift, int64_t d, int64_t S, void* stream,
                          bt_schur* out) {
  if (!out) {
    set_error("bt_schur_create: out is NULL");
    return BT_ERR_ARG;
  }
  *out = nullptr;
  if (nr < 1 || h < 1 || h > 1024 || p < 2 || S < 1 || S > nr || nr % S != 0 || d < -1 || d > 1024 ||
      d >= (p - 1) * nr || !(shift >= 0.0)) {
    set_error("bt_schur_create: need nr >= 1, 1 <= h <= 1024, p >= 2, S | nr, shift >= 0 and "
              "-1 <= d < min(1025, (p - 1) nr)");
    return BT_ERR_ARG;
  }
  bt_schur_s* s = new (std::nothrow) bt_schur_s();
  if (!s) {
    set_error("bt_schur_create: host allocation failed");
    return BT_ERR_OOM;
  }
  cudaGetDevice(&s->device);
  s->nr = nr;
  s->h = h;
  s->p = p;
  s->nz = p * h + p - 1;
  s->ng = (p - 1) * nr;
  s->d = d;
  s->S = S;
  s->shift = shift;
  // preconditioner blocks: at least the half-bandwidth, 16 at the least
  s->MB = std::max<int64_t>(16, d);
  s->SB = std::max<int64_t>(1, std::min<int64_t>(64, (s->ng + s->MB - 1) / s->MB / 4));
  const bt_status rc = build(s, (cudaStream_t)stream);
  if (rc != BT_OK) {
    destroy(s);
    return rc;
  }
  *out = s;
  return BT_OK;
}

void bt_schur_destroy(bt_schur s) { destroy(s); }

bt_status bt_schur_query(bt_schur s, int64_t out[8]) {
  if (!s || !out) {
    set_error("bt_schur_query: NULL argument");
    return BT_ERR_ARG;
  }
  const int64_t v[8] = {s->nr, s->h, s->p, s->nz, s->ng, s->d, s->MB, s->SB};
  std::memcpy(out, v, sizeof(v));
  return BT_OK;
}

bt_status bt_schur_band(bt_schur s, double* ab) {
  if (!s || !ab || !s->ab) {
    set_error("bt_schur_band: need a handle with a preconditioner (d >= 0) and a device buffer");
    return BT_ERR_ARG;
  }
  BT_CUDA(cudaMemcpy(ab, s->ab, (size_t)(2 * s->d + 1) * s->ng * sizeof(double), cudaMemcpyDeviceToDevice));
  return BT_OK;
}

bt_status bt_schur_apply(bt_schur s, const double* v, int64_t K, double* out, void* stream) {
  if (!s || !v || !out || K < 1 || overlap(v, out, (size_t)s->ng * K)) {
    set_error("bt_schur_apply: need a handle, non-overlapping device v and out, K >= 1");
    return BT_ERR_ARG;
  }
  const cudaStream_t st = (cudaStream_t)stream;
  BT_TRY(ensure_k(s, K));
  return apply_S(s, v, K, out, st);
}

bt_status bt_schur_rhs(bt_schur s, const double* F, int64_t K, double* g, void* stream) {
  if (!s || !F || !g || K < 1 || overlap(F, g, (size_t)s->nz * s->nr * K, (size_t)s->ng * K)) {
    set_error("bt_schur_rhs: need a handle, non-overlapping device F and g, K >= 1");
    return BT_ERR_ARG;
  }
  const cudaStream_t st = (cudaStream_t)stream;
  BT_TRY(ensure_k(s, K));
  return reduce_rhs(s, F, K, g, st);
}

bt_status bt_schur_solve(bt_schur s, const double* F, int64_t K, double* X, double tol, int32_t max_it,
                         void* stream, bt_info* info) {
  if (!s || !F || !X || K < 1 || max_it < 0 || !(tol > 0.0)) {
    set_error("bt_schur_solve: need a handle, device F and X, K >= 1, tol > 0, max_it >= 0");
    return BT_ERR_ARG;
  }
  if (overlap(F, X, (size_t)s->nz * s->nr * K)) {
    set_error("bt_schur_solve: X must not overlap F");
    return BT_ERR_ARG;
  }
  const cudaStream_t st = (cudaStream_t)stream;
  BT_TRY(ensure_k(s, K));
  const size_t nv = (size_t)s->ng * K;
  double *g = s->vbuf, *x = g + nv, *r = x + nv, *z = r + nv, *pd = z + nv, *q = pd + nv;
  double *rz = s->cbuf, *rz2 = rz + K, *pq = rz2 + K, *rr = pq + K, *gn2 = rr + K;
  int* active = s->ibuf;
  int* count = s->ibuf + K;
  int* itc = s->ibuf + K + 1;
  const double tol2 = tol * tol;
  // g (eq. schur_decomp, right-hand side), the CG start x = 0, r = g, p = 0
  auto prologue = [&](cudaStream_t st, cudaGraphConditionalHandle loop) -> bt_status {
    BT_TRY(reduce_rhs(s, F, K, g, st));
    BT_CUDA(cudaMemsetAsync(x, 0, nv * sizeof(double), st));
    BT_CUDA(cudaMemsetAsync(pd, 0, nv * sizeof(double), st));
    BT_CUDA(cudaMemcpyAsync(r, g, nv * sizeof(double), cudaMemcpyDeviceToDevice, st));
    BT_TRY(coldot(g, g, s->ng, K, gn2, st));
    k_pcg_init<<<1, 1024, 0, st>>>(rz, K, active, itc);
    k_pcg_check<<<1, 1024, 0, st>>>(gn2, gn2, tol2, K, active, count, itc, max_it, 0, loop);
    BT_CUDA(cudaGetLastError());
    return BT_OK;
  };
  // one PCG iteration: z = B^-1 r, beta = (r, z) / (r, z)_old, p = z + beta p,
  // q = S p, alpha = (r, z) / (p, q), x += alpha p, r -= alpha q, check
  auto body = [&](cudaStream_t st, cudaGraphConditionalHandle loop) -> bt_status {
    BT_TRY(precond(s, r, K, z, st));
    BT_TRY(coldot(r, z, s->ng, K, rz2, st));
    EW(k_pcg_p, nv, pd, z, rz2, rz, active, s->ng, K);
    k_copy_cols<<<(unsigned)((K + 255) / 256), 256, 0, st>>>(rz, rz2, K);
    BT_TRY(apply_S(s, pd, K, q, st));
    BT_TRY(coldot(pd, q, s->ng, K, pq, st));
    EW(k_pcg_xr, nv, x, r, pd, q, rz, pq, active, s->ng, K);
    BT_TRY(coldot(r, r, s->ng, K, rr, st));
    k_pcg_check<<<1, 1024, 0, st>>>(rr, gn2, tol2, K, active, count, itc, max_it, 1, loop);
    BT_CUDA(cudaGetLastError());
    return BT_OK;
  };
  // interiors (eq. domains_equation) and the whole grid panel
  auto epilogue = [&](cudaStream_t st) -> bt_status {
    BT_TRY(strip_solve(s, F, x, K, st));
    EW(k_grid_out, (size_t)s->nz * s->nr * K, strip_out(s, K), x, s->nr, (int)s->h, (int)s->p, K, X);
    return BT_OK;
  };
  // the buffers a captured graph holds (the strip and band solves' own scratch included)
  const std::vector<const void*> ptrs = {s->sbuf, s->vbuf, s->cbuf, s->ibuf, s->strip->scratch,
                                         s->band ? s->band->scratch : nullptr, s->band ? s->band->band_buf : nullptr};
  const bool same = s->pcg_exec && s->pcg_F == F && s->pcg_X == X && s->pcg_K == K && s->pcg_tol == tol &&
                    s->pcg_max == max_it && s->pcg_ptrs == ptrs;
  if (!same) {
    if (s->pcg_exec) cudaGraphExecDestroy(s->pcg_exec);
    s->pcg_exec = nullptr;
    // one direct pass of every sub-solve grows what they allocate on first use,
    // and every kernel of the graph is launched (loaded) once before the capture
    BT_TRY(reduce_rhs(s, F, K, g, st));
    BT_TRY(precond(s, g, K, z, st));
    BT_TRY(apply_S(s, z, K, q, st));
    BT_TRY(coldot(g, g, s->ng, K, gn2, st));
    k_pcg_init<<<1, 1024, 0, st>>>(rz, K, active, itc);
    k_copy_cols<<<(unsigned)((K + 255) / 256), 256, 0, st>>>(rz2, rz, K);
    k_pcg_check<<<1, 1024, 0, st>>>(gn2, gn2, tol2, K, active, count, itc, max_it, 0, 0);
    BT_CUDA(cudaMemsetAsync(pd, 0, nv * sizeof(double), st));
    EW(k_pcg_p, nv, pd, z, rz2, rz, active, s->ng, K);
    EW(k_pcg_xr, nv, x, r, pd, q, rz, pq, active, s->ng, K);
    (void)grid_for((const void*)k_grid_out, (size_t)s->nz * s->nr * K);
    BT_CUDA(cudaStreamSynchronize(st));
    const std::vector<const void*> ptrs2 = {s->sbuf, s->vbuf, s->cbuf, s->ibuf, s->strip->scratch,
                                            s->band ? s->band->scratch : nullptr,
                                            s->band ? s->band->band_buf : nullptr};
    if (!s->cap) BT_CUDA(cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking));
    if (!s->cap2) BT_CUDA(cudaStreamCreateWithFlags(&s->cap2, cudaStreamNonBlocking));
    BT_CUDA(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    bool ok = true;
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    cudaGraphConditionalHandle loop = 0;
    ok = ok && cudaStreamGetCaptureInfo(s->cap, &cs, nullptr, &cg) == cudaSuccess && cg != nullptr;
    ok = ok && cudaGraphConditionalHandleCreate(&loop, cg, 0, cudaGraphCondAssignDefault) == cudaSuccess;
    ok = ok && prologue(s->cap, loop) == BT_OK;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    ok = ok && cudaStreamGetCaptureInfo(s->cap, &cs, nullptr, &cg, &deps, nullptr, &nd) == cudaSuccess;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn = nullptr;
    ok = ok && cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &cp) == cudaSuccess;
    ok = ok && cudaStreamUpdateCaptureDependencies(s->cap, &cn, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                   cudaSuccess;
    if (ok) {
      ok = cudaStreamBeginCaptureToGraph(s->cap2, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const bt_status bs = body(s->cap2, loop);
        cudaGraph_t bg = nullptr;
        ok = cudaStreamEndCapture(s->cap2, &bg) == cudaSuccess && bs == BT_OK;
      }
    }
    ok = ok && epilogue(s->cap) == BT_OK;
    cudaGraph_t graph = nullptr;
    const bool ended = cudaStreamEndCapture(s->cap, &graph) == cudaSuccess;
    // nothing may have moved while capturing (the prepare pass grew every buffer)
    const std::vector<const void*> ptrs3 = {s->sbuf, s->vbuf, s->cbuf, s->ibuf, s->strip->scratch,
                                            s->band ? s->band->scratch : nullptr,
                                            s->band ? s->band->band_buf : nullptr};
    ok = ok && ended && graph && ptrs3 == ptrs2 && cudaGraphInstantiate(&s->pcg_exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
      s->pcg_exec = nullptr;
      const cudaError_t e = cudaGetLastError();
      set_error(std::string("bt_schur_solve: capturing the PCG loop failed: ") + cudaGetErrorString(e));
      return BT_ERR_CUDA;
    }
    s->pcg_F = F;
    s->pcg_X = X;
    s->pcg_K = K;
    s->pcg_tol = tol;
    s->pcg_max = max_it;
    s->pcg_ptrs = ptrs2;
  }
  BT_CUDA(cudaGraphLaunch(s->pcg_exec, st));
  int hc[2] = {0, 0};  // active columns left, iterations
  BT_CUDA(cudaMemcpyAsync(hc, count, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (info) {
    // ||r|| of the last iterate per column (recomputed for columns stopped earlier)
    BT_TRY(coldot(r, r, s->ng, K, rr, st));
    std::vector<double> hrr((size_t)K), hgn((size_t)K);
    BT_CUDA(cudaMemcpyAsync(hrr.data(), rr, (size_t)K * sizeof(double), cudaMemcpyDeviceToHost, st));
    BT_CUDA(cudaMemcpyAsync(hgn.data(), gn2, (size_t)K * sizeof(double), cudaMemcpyDeviceToHost, st));
    BT_CUDA(cudaStreamSynchronize(st));
    double worst = 0.0;
    for (int64_t c = 0; c < K; ++c) worst = std::max(worst, hgn[c] > 0 ? std::sqrt(hrr[c] / hgn[c]) : 0.0);
    info->iters = hc[1];
    info->converged = hc[0] == 0 ? 1 : 0;
    info->rel_res = worst;
    info->rel_res0 = 1.0;
  } else {
    BT_CUDA(cudaStreamSynchronize(st));
  }
  return hc[0] == 0 ? BT_OK : BT_ERR_NOCONV;
}

}  // extern "C"
