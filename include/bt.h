/*
 * bt.h -- C ABI of the block-tridiagonal dichotomy solver (GB300, sm_103a).
 *
 * Solves  -A_j X_{j-1} + C_j X_j - B_j X_{j+1} = F_j,  j = 1..N   (Section 2, eq. main-eq)
 * for many right-hand-side panels against one factored matrix, by the two-stage
 * scheme of Algorithm 2 (Section 2.2): a once-per-matrix preliminary stage
 * (bt_factor) and a per-right-hand-side stage (bt_solve*).
 *
 * Conventions shared by every entry point
 *   - Blocks A, B, C: float64 [N][M][M], row-major, block j at offset j*M*M.
 *     A_1 (index 0) and B_N (index N-1) are not part of the system (the matrix
 *     printed with eq. main-eq has no such entries); their contents are ignored.
 *   - Panels F, X, G, dF: float64 [N][M][K] row-major, i.e. an (N*M) x K matrix
 *     with K contiguous; block row j is the M x K tile at offset j*M*K.
 *   - Unless stated otherwise pointers are DEVICE pointers owned by the caller,
 *     on the CUDA device that is current when the call is made.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Solve calls only enqueue work on it and return; outputs are valid once
 *     the stream has reached that point.
 *   - Errors are reported as bt_status codes only; nothing is thrown across
 *     the ABI.  bt_last_error() gives a human-readable detail string for the
 *     calling thread's most recent failure.
 *   - There is no CPU fallback: every arithmetic step runs in this library's
 *     CUDA kernels; a call on a machine without a usable sm_103 GPU fails
 *     with BT_ERR_CUDA.
 */
#ifndef BT_H_
#define BT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bt_handle_s* bt_handle;

typedef enum {
  BT_OK = 0,
  BT_ERR_ARG = 1,         /* invalid argument (sizes, null pointers, N % S != 0, ...) */
  BT_ERR_SINGULAR = 2,    /* a pivot block of the factorisation is singular or non-finite */
  BT_ERR_CUDA = 3,        /* a CUDA runtime call failed (detail in bt_last_error) */
  BT_ERR_NOCONV = 4,      /* iterative refinement did not reach the requested tolerance */
  BT_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  BT_ERR_OOM = 6,         /* device memory allocation failed */
  BT_ERR_UNSUPPORTED = 7  /* valid request that the library does not implement */
} bt_status;

typedef enum {
  BT_PREC_F64 = 0,   /* every product in FP64 */
  BT_PREC_TF32 = 1,  /* panel products on tensor cores in TF32, FP32 accumulation */
  BT_PREC_BF16 = 2,  /* panel products on tensor cores in BF16, FP32 accumulation */
  BT_PREC_F32 = 3,   /* panel products on the CUDA cores in FP32 */
  BT_PREC_BF16X3 = 4 /* tensor cores, every operand split into two BF16 terms (hi + lo),
                        three MMAs per product: about 2^-17 relative operand precision */
} bt_precision;

/* Options of bt_solve_ex.  Zero-initialised options mean: FP64, defaults. */
typedef struct {
  int32_t precision;  /* bt_precision */
  int32_t max_it;     /* refinement passes after the first solve (0 = default: 6 for
                         BT_PREC_BF16X3, 12 otherwise) */
  double tol;         /* target ||F - P X||_F / ||F||_F (0 = default 1e-10) */
  void* stream;       /* cudaStream_t */
  int32_t k_tile;     /* right-hand-side columns per CTA (0 = automatic) */
  int32_t residual;   /* how F - P X is formed: 0 automatic (2 or 3 where they
                         apply, else 1), 1 FP64 on the CUDA cores, 2 exactly on
                         the tensor cores from BF16 digit slices (dense blocks,
                         M = 64 or 128), 3 in FP32 double-word arithmetic (unit
                         stencils: see bt_residual); BT_ERR_UNSUPPORTED where
                         2 or 3 does not apply */
} bt_opts;

/* Result report of bt_solve_ex (filled only when a non-NULL pointer is given;
 * the call then synchronises its stream before returning). */
typedef struct {
  int32_t iters;      /* refinement passes performed after the first solve */
  int32_t converged;  /* 1 if rel_res <= tol */
  double rel_res;     /* final ||F - P X||_F / ||F||_F, measured in FP64 */
  double rel_res0;    /* the same after the first (unrefined) solve */
} bt_info;

/*
 * bt_factor -- Algorithm 2, stage 1 (Section 2.2, steps 1.1-1.3), all in FP64
 * on the GPU:
 *   1.1  per segment, the block-sweep factorisation of the interior rows and
 *        the coupling responses U, V of eqs. sub1 / sub2;
 *   1.2  the reduced (interface) system of eq. red1;
 *   1.3  the stored block rows of the inverses needed by Algorithm 1 on it.
 * N   block rows (>= 1); M block size (1..1024; tested up to 256); S segments, 1 <= S <= N and
 *     N % S == 0 (the paper's L = N/p); interface rows are 1, L+1, ..., (S-1)L+1.
 * A, B, C  device pointers as described above; they are only read, and may be
 *     freed once this call returns.
 * out receives a handle that owns all factor memory on the current device.
 * The products with A_j and B_j run over the diagonals that hold their
 * nonzero entries only (found by a scan of A and B; see bt_handle_band), which
 * gives the same values as full products.
 * The call synchronises `stream` twice: to read those bands before the
 * factorisation is scheduled, and to read the pivot status at the end:
 *   BT_ERR_SINGULAR if any pivot block is singular or non-finite (no handle
 *   is returned), BT_ERR_ARG for invalid sizes or NULL pointers,
 *   BT_ERR_OOM / BT_ERR_CUDA on device failures.
 */
bt_status bt_factor(int64_t N, int64_t M, const double* A, const double* B, const double* C,
                    int64_t S, void* stream, bt_handle* out);

/*
 * bt_factor_band -- bt_factor for a band matrix (Section 3.3.1, item c: the PML
 * operator A_44, a band matrix solved by the dichotomy as a block-tridiagonal
 * matrix with triangular off-diagonal blocks).
 * Q: order n, kl sub-diagonals and ku super-diagonals (0 <= kl, ku <= M), in
 *   diagonal-ordered storage: ab is a DEVICE (kl + ku + 1) x n row-major FP64
 *   array with ab[(ku + i - j) * n + j] = Q[i][j] for -ku <= i - j <= kl
 *   (the other positions of ab are not read).  Read only; may be freed when
 *   the call returns.
 * M: block size; S: segments.  The system is cut into N = S ceil(ceil(n/M)/S)
 *   block rows of M rows (rows and columns n .. N M - 1 padded with the
 *   identity), so that C_j = Q[jM.., jM..], A_j = -Q[jM.., (j-1)M..] (upper
 *   triangular) and B_j = -Q[jM.., (j+1)M..] (lower triangular) in the sign
 *   convention of bt_factor.  Needs 1 <= S <= ceil(n / M).
 * The factorisation detects the bands of A_j and B_j (any bt_factor does) and
 * runs its products with A_j and B_j over the nonzero diagonals only.
 * Temporary device memory: the three block arrays (3 N M^2 doubles), released
 * before return.  Errors as bt_factor.  Solve with bt_solve_band (or, when
 * n = N M, with any bt_solve* call on (n x K) panels).
 */
bt_status bt_factor_band(int64_t n, int64_t kl, int64_t ku, const double* ab, int64_t M, int64_t S,
                         void* stream, bt_handle* out);

/*
 * bt_solve_band -- bt_solve_ex on a handle of bt_factor_band: F and X are
 * DEVICE n x K row-major FP64 panels (X must not overlap F); opts and info as
 * bt_solve_ex (opts->stream carries the work).  When n < N M the call pads F
 * with zero rows into a panel pair owned by the handle (grown on demand) and
 * copies the first n rows of the solution to X.  BT_ERR_ARG on a handle not
 * made by bt_factor_band; BT_ERR_NOCONV still writes the last iterate to X.
 */
bt_status bt_solve_band(bt_handle h, const double* F, int64_t K, double* X, const bt_opts* opts,
                        bt_info* info);

/*
 * bt_solve -- Algorithm 2, stage 2 (Section 2.2, steps 2.1-2.3) in FP64:
 *   2.1  per-segment sweeps of eq. sub3 (W),
 *   2.2  Algorithm 1 on the reduced system eq. red1 (interface unknowns),
 *   2.3  every row from eq. superposition.
 * F  device [N][M][K] right-hand sides (read only); X device [N][M][K] output.
 * X must not overlap F.  K >= 1.  Asynchronous on `stream`.
 * Scratch memory is taken from a pool owned by the handle (grown on demand);
 * concurrent calls on one handle must use the same stream.
 */
bt_status bt_solve(bt_handle h, const double* F, int64_t K, double* X, void* stream);

/*
 * bt_solve_ex -- stage 2 with a selectable precision.  BT_PREC_F64 is
 * bt_solve.  BT_PREC_TF32 / BT_PREC_BF16 run the panel products of steps
 * 2.1-2.3 on tcgen05 tensor cores with FP32 accumulation against rounded
 * copies of the factors (BT_PREC_F32: FP32 on the CUDA cores), and recover
 * FP64 accuracy by iterative refinement against the residual F - P X formed
 * to FP64 accuracy (not in the paper): X_0 = S~ F,
 * X_{k+1} = X_k + S~ (F - P X_k), until ||F - P X||_F <= tol ||F||_F or
 * max_it passes.  F, X, K as for bt_solve.  When `info` is non-NULL the call
 * synchronises the stream and fills it; with info == NULL it is asynchronous
 * and never returns BT_ERR_NOCONV.  The residual is formed per opts->residual
 * (see bt_opts; for dense blocks with M = 64 or 128 exactly on the tensor
 * cores by default).  The tensor-core precisions take block sizes M <= 128:
 * below the tiles (64, 128) the factor blocks, interface blocks and internal
 * panels are padded with zero rows and columns, whose unknowns stay zero
 * (BT_ERR_UNSUPPORTED past 128).  The handle keeps the refinement as CUDA graphs, one per
 * argument key (F, X, K, precision, tol, max_it, residual method; at most 64,
 * least recently used out, dropped when a refinement buffer is reallocated): a
 * key's second call captures, later calls replay.  Calls on one handle must be
 * ordered on one stream; different handles may run concurrently.
 */
bt_status bt_solve_ex(bt_handle h, const double* F, int64_t K, double* X, const bt_opts* opts,
                      bt_info* info);

/*
 * bt_solve_host -- bt_solve_ex for right-hand sides in host memory (not in the
 * paper): F and X are HOST [N][M][K] FP64 arrays (page-locked for the copies
 * to overlap; pageable memory works, synchronously).  The columns go through
 * the device in chunks of 128 (at least about four chunks per call): the upload
 * of a chunk, the solve of the previous one (on opts->stream) and the download
 * of the one before run concurrently, in two device panel pairs owned by the
 * handle (grown on demand; each pair keeps its own CUDA graph).  Synchronous:
 * X is complete on return.  No bt_info (as bt_solve_ex with info == NULL).
 */
bt_status bt_solve_host(bt_handle h, const double* F, int64_t K, double* X, const bt_opts* opts);

/*
 * bt_solve_adjoint -- gradients of a loss through X = P^{-1} F (not in the
 * paper).  With G = dL/dX, solves P^T lambda = G by the same stage-2 machinery
 * on the factors of P^T (built on first use and kept in the handle) and forms
 *   dF = lambda,  dC_j = -lambda_j X_j^T,  dA_j = lambda_j X_{j-1}^T (j > 1),
 *   dB_j = lambda_j X_{j+1}^T (j < N),  dA_1 = dB_N = 0,
 * each summed over the K columns.  X: the solution [N][M][K]; G: [N][M][K];
 * dF: [N][M][K]; dA, dB, dC: [N][M][M] (any of the four outputs may be NULL).
 * All device pointers, FP64.  Asynchronous on `stream`, except that the first
 * call on a handle factors P^T and synchronises once.
 */
/*
 * bt_residual -- r = F - P X for the factored operator (eq. (1) with the
 * blocks given to bt_factor), the quantity the refinement of bt_solve_ex
 * drives to zero; the paper has no counterpart.  F, X: device [N][M][K]
 * (read only); R: device [N][M][K] output (may alias neither).  method:
 *   0  automatic (2 where it applies, else 1),
 *   1  FP64 on the CUDA cores,
 *   2  on the tensor cores: every value of the operator rows and of X is
 *      split into seven balanced base-128 digits (one power-of-two scale per
 *      operator row, one per column of X), the digit products are summed
 *      exactly in FP32, and the sums are combined with F in 64-bit integer
 *      arithmetic.  Error per entry at most 7.5 M 2^(e_A + e_X - 49), e_A and
 *      e_X the scales (2^e_A > the row's largest |A|, |B|, |C| entry, 2^e_X >
 *      the column's largest |X| entry).  Dense blocks with M = 64 or 128 only
 *      (BT_ERR_UNSUPPORTED otherwise).
 *   3  in FP32 arithmetic on the CUDA cores, for unit stencils: A_j = B_j = I
 *      and C_j = tridiag(-1, c, -1) with 2^-30 <= |c| <= 2^30, M a multiple
 *      of 8 (BT_ERR_UNSUPPORTED otherwise).  Every FP64 value is split into
 *      two FP32 terms (24 + 23 bits), the unit-coefficient terms are summed
 *      exactly (TwoSum), c x enters through one FMA and the low-order terms
 *      are summed in FP32; the result is an FP32 value per entry (stored in
 *      R as FP64).  Error per entry at most 2^-23 |r| + 2^-42 S with
 *      S = |f| + |x_{j-1}| + |x_{j+1}| + |x_{m-1}| + |x_{m+1}| + |c x|;
 *      values below 2^-100 in magnitude count as zero.  If any value of F or
 *      X is 2^77 or larger in magnitude (or not finite) the residual is
 *      recomputed by method 1.
 * norm2 (host, may be NULL) receives ||r||_F^2.  Synchronises `stream`.
 */
bt_status bt_residual(bt_handle h, const double* F, const double* X, int64_t K, double* R, int32_t method,
                      double* norm2, void* stream);

bt_status bt_solve_adjoint(bt_handle h, const double* X, const double* G, int64_t K, double* dF,
                           double* dA, double* dB, double* dC, void* stream);

/*
 * Batched solves (not in the paper): many right-hand-side sets, each against
 * one of a few factored matrices, planned once and run as ONE CUDA graph
 * launch.
 *   - FP64 plans (opts->precision BT_PREC_F64): one persistent cooperative
 *     launch runs stage 2 of Algorithm 2 for all sets -- sweeps, interface
 *     terms, one stage per dichotomy level, corrections, separated by
 *     grid-wide barriers.
 *   - Refined plans (any other precision): stage 2 is linear in F and its
 *     factors do not depend on F, so the sets of each matrix are packed side
 *     by side into one panel and solved by ONE refined solve (bt_solve_ex) per
 *     matrix; the matrices run on concurrent branches of the graph and every
 *     refinement loop is a device-side WHILE node.  Set s is scaled by the
 *     power of two 2^-e_s with 2^(e_s-1) <= ||F_s||_F < 2^e_s before packing
 *     (exact), and the packed refinement runs until EVERY set meets
 *     ||F_s - P X_s||_F <= tol ||F_s||_F on its own, as if solved alone
 *     (each set's sum of squares is taken from the residual panel after
 *     every pass, with a margin for the panel's rounding).  The packed panels
 *     (2 N M sum(K) doubles per matrix) are
 *     owned by the plan.
 *
 * bt_batch_create -- plans a batch of n >= 1 sets; set i solves
 *   P_{h[i]} X_i = F_i, F[i] and X[i] being device [N_i][M][K[i]] FP64 panels
 *   as for bt_solve.  h, F, K, X are HOST arrays of n entries; the panels are
 *   device memory owned by the caller that must keep their addresses while
 *   the plan is used (the plan records the pointers).  All handles live on the
 *   current device and share one block size M (N and S may differ).  No X[i]
 *   may overlap an F[j] or another X[j].  opts (may be NULL): precision,
 *   tol, max_it and residual as for bt_solve_ex (refined plans; at most 1024
 *   sets per matrix); k_tile = right-hand-side columns per work item of the
 *   FP64 launch (0 = automatic); stream is not used.  The plan owns its
 *   scratch and its graph; the handles must outlive it, and no other call may
 *   use a handle of a refined plan while the plan runs (they share the
 *   handle's refinement scratch).  Synchronous; BT_ERR_ARG on invalid input,
 *   BT_ERR_UNSUPPORTED where bt_solve_ex would refuse the precision or
 *   residual for a handle.
 * bt_batch_run -- enqueues one batched solve on `stream` (one graph launch).
 *   A refined plan whose handles' refinement scratch was reallocated by a
 *   later call with more columns is prepared and captured again first
 *   (synchronous, allocating).
 * bt_batch_status -- waits for the plan's work and returns BT_OK, or
 *   BT_ERR_TIMEOUT if a bounded wait of the last run gave up (FP64: a
 *   grid-barrier wait, 20 s by default, see bt_batch_debug; refined: a
 *   tensor-core wait), or BT_ERR_NOCONV if a refined matrix group did not reach
 *   its tolerance within max_it passes.  The device stays usable: the plan can
 *   be run again.
 * bt_batch_info -- after bt_batch_status: the refinement report of set i's
 *   matrix group (iters, converged -- every set of the group met tol -- and
 *   rel_res / rel_res0 of the packed, scaled panel as a whole); FP64 plans
 *   report iters 0, converged 1, rel_res -1.
 * bt_batch_debug -- diagnostics for testing the failure path of FP64 plans
 *   (BT_ERR_UNSUPPORTED for refined plans): limit_s sets the grid-barrier wait
 *   limit of later runs (0 = the 20 s default, at most 60 s); skip_stage >= 0
 *   plants a failure -- CTA 0 of the persistent launch leaves the kernel
 *   instead of arriving at the barrier after that stage, so the other CTAs'
 *   waits run out and the run reports BT_ERR_TIMEOUT; -1 removes it.  Takes
 *   effect in graph replays too.  Synchronises the device.
 * bt_batch_query -- FP64 plans: out[0] work items, out[1] stages, out[2] CTAs
 *   of the persistent launch, out[3] threads per CTA, out[4] columns per item;
 *   refined plans: out[0] matrix groups (packed panels), out[1..3] 0, out[4]
 *   the k_tile option; out[5] 1 when runs replay a CUDA graph.
 * bt_solve_batched -- create, run on opts->stream, wait, destroy.
 */
typedef struct bt_batch_s* bt_batch;
bt_status bt_batch_create(int32_t n, const bt_handle* h, const double* const* F, const int64_t* K,
                          double* const* X, const bt_opts* opts, bt_batch* out);
bt_status bt_batch_run(bt_batch b, void* stream);
bt_status bt_batch_status(bt_batch b);
bt_status bt_batch_query(bt_batch b, int64_t out[6]);
bt_status bt_batch_info(bt_batch b, int32_t i, bt_info* out);
bt_status bt_batch_debug(bt_batch b, double limit_s, int32_t skip_stage);
void bt_batch_destroy(bt_batch b);
bt_status bt_solve_batched(int32_t n, const bt_handle* h, const double* const* F, const int64_t* K,
                           double* const* X, const bt_opts* opts);

/*
 * bt_solve_noalloc -- the FP64 solve of bt_solve, for callers that cannot
 * allocate device memory at solve time.  The paper has no counterpart: it is a
 * service of this library.  Some callers cannot call cudaMalloc once they are
 * running: a host whose device memory is owned by another allocator (a
 * framework's caching pool or a fixed arena), or a latency-bound loop that
 * must not take the device-wide synchronisation cudaMalloc and cudaFree may
 * imply.  bt_solve grows a scratch buffer in the handle on first use;
 * this entry point instead uses a scratch array of BT_NOALLOC_SCRATCH_BYTES
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits.
 *   - F, K, X, stream: as for bt_solve (the caller owns inputs and outputs).
 *   - The scratch needed is depth * S * M * K * 8 bytes (depth from
 *     bt_handle_query); larger requests (and K < 1) return BT_ERR_ARG and do
 *     nothing.  The check divides instead of multiplying, so no K wraps it.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) for that device; make that first call before any
 *     stream capture.  The device of the handle must be current.  The address
 *     is kept per device together with the CUDA context it was found in; a
 *     call in another context (after a device reset) looks it up again -- and
 *     should again come before any stream capture.
 *   - All calls share the one array per device: calls whose work overlaps on
 *     the GPU (other streams, other threads) race on it and give wrong results.
 *     The array keeps the previous call's contents; this solve overwrites
 *     every entry it reads, so nothing needs clearing.
 *   - No cudaMalloc, cudaFree or other allocating routine is called.
 */
#define BT_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
bt_status bt_solve_noalloc(bt_handle h, const double* F, int64_t K, double* X, void* stream);

/* Releases the handle and all its device memory (synchronises the device). */
void bt_destroy(bt_handle h);

/* Static description of a status code. */
const char* bt_strerror(bt_status s);

/* Detail of the calling thread's most recent failure ("" if none). */
const char* bt_last_error(void);

/*
 * bt_handle_query -- sizes of a factored handle.
 * out[0] = N, out[1] = M, out[2] = S, out[3] = depth of the dichotomy tree,
 * out[4] = 1 if the matrix has A_j = B_j = I and tridiagonal C_j (a stencil
 * operator), else 0, out[5] = device bytes held by the handle.
 */
bt_status bt_handle_query(bt_handle h, int64_t out[6]);

/*
 * Schur-complement CG with a probing band preconditioner (Section 3.3: the
 * interface system of eq. schur_decomp solved by CG without forming S, the
 * interiors by eq. domains_equation; Section 3.3.2: the probing band
 * preconditioner B, inverted by the dichotomy).
 * Model problem: the five-point operator (4 + shift) x_{z,r} - x_{z-1,r} -
 * x_{z+1,r} - x_{z,r-1} - x_{z,r+1} (zero values outside) on an nz x nr grid,
 * cut by p - 1 interface grid rows into p strips of h rows: nz = p h + p - 1,
 * strip i holds rows i (h + 1) .. i (h + 1) + h - 1, interface line k is row
 * k (h + 1) + h.  Each strip operator, unknowns ordered by grid column, is a
 * block-tridiagonal system with N = nr blocks of M = h (A_j = B_j = I,
 * C_j = tridiag(-1, 4 + shift, -1)); the strips share one factorisation (S
 * segments) and are solved together, p K columns per dichotomy solve.
 * Panels: grid F, X [nz][nr][K]; interface v, g [p - 1][nr][K] (ng = (p-1) nr
 * rows); all FP64 device arrays, K contiguous.
 */
typedef struct bt_schur_s* bt_schur;

/*
 * bt_schur_create -- factors the strip operator and builds the preconditioner:
 * one product of S with the 2d+1 probing vectors (1 on the interface indices
 * congruent to l modulo 2d+1), B[i][j] = (S p_{j mod (2d+1)})[i] for
 * |i - j| <= d, symmetrised ((B + B^T) / 2; S is symmetric), factored by
 * bt_factor_band with blocks of max(16, d) rows.  d = -1: no preconditioner.
 * Needs nr >= 1, 1 <= h <= 1024, p >= 2, nr % S == 0, shift >= 0 and
 * -1 <= d < min(1025, ng).  Synchronises `stream`.  Errors as bt_factor.
 */
bt_status bt_schur_create(int64_t nr, int64_t h, int64_t p, double shift, int64_t d, int64_t S, void* stream,
                          bt_schur* out);

/* S v for an interface panel v (K columns) into out (must not overlap v); asynchronous. */
bt_status bt_schur_apply(bt_schur s, const double* v, int64_t K, double* out, void* stream);

/* g = f_G - sum_i A_Gi A_ii^{-1} f_i for a grid panel F (eq. schur_decomp) into an interface
 * panel g (must not overlap F); asynchronous. */
bt_status bt_schur_rhs(bt_schur s, const double* F, int64_t K, double* g, void* stream);

/*
 * bt_schur_solve -- X = A^{-1} F for a grid panel F: g, then preconditioned CG
 * (Saad, Algorithm 9.1) on S x_G = g for all K columns at once from x_G = 0,
 * a column stopping once ||g - S x_G|| <= tol ||g|| (the recursively updated
 * residual), at most max_it iterations; then the interiors (eq.
 * domains_equation) and X.  Each iteration: one product with S (one
 * dichotomy solve of p K columns), one solve with B, three column dot
 * products and the convergence check.  The whole solve is one CUDA graph: the
 * iterations are the body of a device-side WHILE node whose condition the
 * check sets (active columns remain, fewer than max_it iterations), so the
 * host does not wait per iteration.  A call with new arguments (F, X, K, tol,
 * max_it) or after a buffer moved first runs every sub-solve once directly and
 * captures the graph (synchronous); repeated calls replay it.  The call
 * synchronises `stream` once at the end.  X must not overlap F.  info (may be NULL): iterations,
 * converged, rel_res = the largest relative residual over the columns,
 * rel_res0 = 1.  BT_ERR_NOCONV if a column did not converge (X is then the
 * solution for the last iterate).
 */
bt_status bt_schur_solve(bt_schur s, const double* F, int64_t K, double* X, double tol, int32_t max_it,
                         void* stream, bt_info* info);

/* Copies B (band storage [2d+1][ng], ab[d + i - j][j] = B[i][j]) to a device buffer; synchronous. */
bt_status bt_schur_band(bt_schur s, double* ab);

/* out = {nr, h, p, nz, ng, d, block size of B, segments of B}. */
bt_status bt_schur_query(bt_schur s, int64_t out[8]);

/* Releases the handle (synchronises the device). */
void bt_schur_destroy(bt_schur s);

/*
 * bt_handle_band -- the diagonal bands the factorisation found and used:
 * out[0..1] = smallest and largest c - r over the nonzero entries (r, c) of
 * A_j (j > 1), out[2..3] the same for B_j (j < N) (0, 0 for an all-zero
 * operator; -(M-1), M-1 for a dense one), out[4] = n for a handle of
 * bt_factor_band, else 0.
 */
bt_status bt_handle_band(bt_handle h, int64_t out[5]);

/*
 * bt_factor_export -- copies one FP64 array of the factorisation into a
 * caller-owned device buffer (diagnostics and step-wise verification).
 *   what = 0: U  [N][M][M]   coupling response of eq. sub1 on interior rows
 *   what = 1: V  [N][M][M]   coupling response of eq. sub2 on interior rows
 *   what = 2: At [S][M][M]   reduced system of eq. red1, sub-diagonal blocks
 *   what = 3: Ct [S][M][M]   reduced system, diagonal blocks
 *   what = 4: Bt [S][M][M]   reduced system, super-diagonal blocks
 *   what = 5: Y  [N][M][M]   forward responses of the left coupling on
 *                            interior rows, Y_a = E_a, Y_i = E_i Y_{i-1} with
 *                            E_i = D_i^{-1} A_i (the first half of eq. sub1;
 *                            built on first use)
 * Rows that are interfaces hold zeros in U, V and Y.  Synchronous.
 */
bt_status bt_factor_export(bt_handle h, int32_t what, double* dst);

/*
 * bt_solve_stages -- runs only the first `stages` steps of bt_solve's FP64
 * pipeline (diagnostics and step-wise verification):
 *   stages = 1: X holds W of eq. sub3 on interior rows (step 2.1);
 *   stages = 2: additionally X holds X~ of eq. red1 on interface rows (step 2.2);
 *   stages = 3: the full solution (step 2.3), identical to bt_solve.
 * Rows not yet written are left untouched.  Asynchronous on `stream`.
 */
bt_status bt_solve_stages(bt_handle h, const double* F, int64_t K, double* X, int32_t stages,
                          void* stream);

/*
 * Per-kernel timing (diagnostics for the benchmark; not in the paper).
 * bt_profile_enable(h, 1) makes every later launch on this handle record a
 * CUDA event pair on its stream around each kernel; 0 stops recording.
 * bt_profile_read synchronises the recorded events, writes up to `cap`
 * per-kernel totals (launch count and summed device time in milliseconds,
 * grouped by kernel name) to `out`, sets *n to the number of kernel names and
 * clears the totals.  Timing adds two event records per launch.
 */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
} bt_kernel_stat;

bt_status bt_profile_enable(bt_handle h, int32_t enable);
bt_status bt_profile_read(bt_handle h, bt_kernel_stat* out, int32_t cap, int32_t* n);

#ifdef __cplusplus
}
#endif

#endif /* BT_H_ */
