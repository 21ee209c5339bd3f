// Gradients through X = P^{-1} F (not in the paper).
//
// For a loss L(X) with G = dL/dX: lambda = P^{-T} G, dL/dF = lambda and
// dL/dP = -lambda X^T.  P holds -A_j, C_j, -B_j (eq. main-eq), so with the K
// right-hand sides summed:
//   dC_j = -lambda_j X_j^T,  dA_j = lambda_j X_{j-1}^T (j > 1),
//   dB_j =  lambda_j X_{j+1}^T (j < N),  dA_1 = dB_N = 0.
// P^T is block tridiagonal with A'_j = B_{j-1}^T, B'_j = A_{j+1}^T,
// C'_j = C_j^T; it is factored on first use with the same stage-1 code and
// kept in the handle, and lambda comes from the same stage-2 kernels.

#include "bt_internal.cuh"

namespace bt {

namespace {

// Blocks of P^T from the handle's copies of A, B, C.
__global__ void k_transpose_blocks(const double* __restrict__ A, const double* __restrict__ B,
                                   const double* __restrict__ C, double* __restrict__ At, double* __restrict__ Bt,
                                   double* __restrict__ Ct, int64_t N, int M) {
  const size_t MM = (size_t)M * M, n = (size_t)N * MM;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t j = e / MM;
    const int r = (int)((e % MM) / M), c = (int)(e % M);
    const size_t tr = (size_t)c * M + r;  // transposed position inside a block
    Ct[e] = C[j * MM + tr];
    At[e] = j > 0 ? B[(j - 1) * MM + tr] : 0.0;
    Bt[e] = j + 1 < N ? A[(j + 1) * MM + tr] : 0.0;
  }
}

// out_j (M x M) = sign * lam_j (M x K) * Y_{j+shift}^T (K x M), FP64; a block
// row without a partner (j+shift outside 0..N-1) gets zeros.  32 x 32 output
// tile per CTA, 256 threads with 2 x 2 outputs each, K staged 32 at a time.
__global__ void __launch_bounds__(256) k_adj_grad(const double* __restrict__ lam, const double* __restrict__ Y,
                                                  double* __restrict__ out, int64_t N, int M, int64_t K,
                                                  int shift, double sign) {
  __shared__ double ls[32][33];
  __shared__ double ys[32][33];
  const int64_t j = blockIdx.z;
  const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t jp = j + shift;
  const bool has = jp >= 0 && jp < N;
  const size_t MK = (size_t)M * K;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  if (has) {
    const double* L = lam + j * MK;
    const double* Yp = Y + jp * MK;
    for (int64_t k0 = 0; k0 < K; k0 += 32) {
      for (int e = threadIdx.x; e < 32 * 32; e += 256) {
        const int r = e / 32, c = e % 32;
        const int64_t k = k0 + c;
        ls[r][c] = (a0 + r < M && k < K) ? L[(size_t)(a0 + r) * K + k] : 0.0;
        ys[r][c] = (b0 + r < M && k < K) ? Yp[(size_t)(b0 + r) * K + k] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < 32; ++kk) {
        const double l0 = ls[ty * 2][kk], l1 = ls[ty * 2 + 1][kk];
        const double y0 = ys[tx * 2][kk], y1 = ys[tx * 2 + 1][kk];
        acc[0][0] = fma(l0, y0, acc[0][0]);
        acc[0][1] = fma(l0, y1, acc[0][1]);
        acc[1][0] = fma(l1, y0, acc[1][0]);
        acc[1][1] = fma(l1, y1, acc[1][1]);
      }
      __syncthreads();
    }
  }
  for (int i = 0; i < 2; ++i)
    for (int k = 0; k < 2; ++k) {
      const int a = a0 + ty * 2 + i, b = b0 + tx * 2 + k;
      if (a < M && b < M) out[j * (size_t)M * M + (size_t)a * M + b] = sign * acc[i][k];
    }
}

}  // namespace

bt_status make_handle(int64_t N, int64_t M, const double* A, const double* B, const double* C, int64_t S,
                      cudaStream_t st, bt_handle_s** out);

bt_status solve_adjoint(bt_handle_s* h, const double* X, const double* G, int64_t K, double* dF, double* dA,
                        double* dB, double* dC, cudaStream_t st) {
  const int M = (int)h->M;
  const size_t MM = (size_t)M * M;
  if (!h->adj) {
    double *At = nullptr, *Bt = nullptr, *Ct = nullptr;
    const size_t bytes = h->N * MM * sizeof(double);
    BT_CUDA(cudaMalloc(&At, bytes));
    BT_CUDA(cudaMalloc(&Bt, bytes));
    BT_CUDA(cudaMalloc(&Ct, bytes));
    k_transpose_blocks<<<1024, 256, 0, st>>>(h->A, h->B, h->C, At, Bt, Ct, h->N, M);
    bt_status s = cudaGetLastError() == cudaSuccess ? BT_OK : BT_ERR_CUDA;
    if (s == BT_OK) s = make_handle(h->N, h->M, At, Bt, Ct, h->S, st, &h->adj);
    cudaStreamSynchronize(st);
    cudaFree(At);
    cudaFree(Bt);
    cudaFree(Ct);
    if (s != BT_OK) {
      h->adj = nullptr;
      return s;
    }
  }
  // lambda = P^{-T} G, into dF when the caller wants it, else into the handle's buffer
  double* lam = dF;
  if (!lam) {
    const size_t need = (size_t)h->N * M * K * sizeof(double);
    if (need > h->adj_lam_bytes) {
      if (h->adj_lam) {
        BT_CUDA(cudaStreamSynchronize(st));
        BT_CUDA(cudaFree(h->adj_lam));
      }
      h->adj_lam = nullptr;
      h->adj_lam_bytes = 0;
      BT_CUDA(cudaMalloc(&h->adj_lam, need));
      h->adj_lam_bytes = need;
    }
    lam = reinterpret_cast<double*>(h->adj_lam);
  }
  BT_TRY(solve_f64(h->adj, G, K, lam, 3, st));
  const dim3 grid((M + 31) / 32, (M + 31) / 32, (unsigned)h->N);
  {
    ProfScope ps(h, st, "adj_grad");
    if (dC) k_adj_grad<<<grid, 256, 0, st>>>(lam, X, dC, h->N, M, K, 0, -1.0);
    if (dA) k_adj_grad<<<grid, 256, 0, st>>>(lam, X, dA, h->N, M, K, -1, 1.0);
    if (dB) k_adj_grad<<<grid, 256, 0, st>>>(lam, X, dB, h->N, M, K, +1, 1.0);
  }
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

}  // namespace bt
