// Band matrices as block-tridiagonal systems (Section 3.3.1, item c: the PML
// operator A_44 is a band matrix that the dichotomy solves as a block-
// tridiagonal one with triangular off-diagonal blocks).
//
// A band matrix Q of order n with kl sub- and ku super-diagonals (kl, ku <= M)
// is cut into N = S * ceil(ceil(n / M) / S) block rows of M rows; rows and
// columns n .. N*M-1 are padded with the identity.  Block row j of the system
//   -A_j X_{j-1} + C_j X_j - B_j X_{j+1} = F_j
// then holds C_j = Q[jM.., jM..], A_j = -Q[jM.., (j-1)M..], B_j = -Q[jM..,
// (j+1)M..] (the sign convention of the block equation).  Entry (r, c) of A_j
// can be nonzero only where c - r >= M - kl (upper triangular) and of B_j
// only where c - r <= ku - M (lower triangular); the factorisation detects
// those bands and shortens the GEMM contractions they allow.
#include "bt_internal.cuh"

namespace bt {

namespace {

// Q[i][col] from the diagonal-ordered band storage ab[(ku + i - col) * n + col];
// the identity beyond the order n.
__device__ __forceinline__ double band_entry(const double* __restrict__ ab, int64_t n, int64_t kl, int64_t ku,
                                             int64_t i, int64_t col) {
  if (i >= n || col >= n) return i == col ? 1.0 : 0.0;
  const int64_t d = i - col;
  if (d > kl || -d > ku) return 0.0;
  return ab[(ku + d) * n + col];
}

// One thread per entry of the block arrays (writes coalesced; the band is
// gathered through L2).
__global__ void k_band_to_blocks(const double* __restrict__ ab, int64_t n, int64_t kl, int64_t ku, int64_t N,
                                 int M, double* __restrict__ A, double* __restrict__ B, double* __restrict__ C) {
  const size_t MM = (size_t)M * M, tot = (size_t)N * MM;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t j = (int64_t)(e / MM);
    const size_t w = e - (size_t)j * MM;
    const int64_t r = (int64_t)(w / M), c = (int64_t)(w % M);
    const int64_t i = j * M + r;
    C[e] = band_entry(ab, n, kl, ku, i, j * M + c);
    const double a = j > 0 ? band_entry(ab, n, kl, ku, i, (j - 1) * M + c) : 0.0;
    const double b = j < N - 1 ? band_entry(ab, n, kl, ku, i, (j + 1) * M + c) : 0.0;
    A[e] = a == 0.0 ? 0.0 : -a;
    B[e] = b == 0.0 ? 0.0 : -b;
  }
}

}  // namespace

bt_status band_to_blocks(const double* ab, int64_t n, int64_t kl, int64_t ku, int64_t N, int64_t M, double* A,
                         double* B, double* C, cudaStream_t st) {
  const size_t tot = (size_t)N * M * M;
  const int grid = (int)std::min<size_t>((tot + 255) / 256, (size_t)resident_grid((const void*)k_band_to_blocks, 256, 0));
  k_band_to_blocks<<<std::max(grid, 1), 256, 0, st>>>(ab, n, kl, ku, N, (int)M, A, B, C);
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

}  // namespace bt
