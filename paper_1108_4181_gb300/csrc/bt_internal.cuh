// Internal declarations shared by the CUDA translation units of libbt.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bt.h"

namespace bt {

// ---------------------------------------------------------------------------
// Error handling: status codes only cross the ABI; details go to a
// thread-local string read by bt_last_error().
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
bt_status cuda_fail(cudaError_t e, const char* what);

#define BT_CUDA(call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return ::bt::cuda_fail(e_, #call);  \
  } while (0)

#define BT_TRY(call)                        \
  do {                                      \
    bt_status s_ = (call);                  \
    if (s_ != BT_OK) return s_;             \
  } while (0)

// A node of the dichotomy tree over the S interface unknowns (Algorithm 1 on
// the reduced system): sub-range [l, r], middle unknown m, tree level.
struct TreeNode {
  int l, r, m, level;
};

// Dichotomy tree with the split m = l + (r - l) / 2, breadth first.
std::vector<TreeNode> build_tree(int S, int* depth_out);

// Per-kernel CUDA-event timing, enabled per handle (bt_profile_enable).
struct Profiler {
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
  };
  bool on = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  std::vector<std::string> names;
  std::vector<int64_t> launches;
  std::vector<double> total_ms;
  cudaEvent_t get();
  void collect();   // synchronises pending records into the totals
  void destroy();
};

// Device memory owned by a handle: a list of allocations freed together.
struct DevArena {
  std::vector<void*> blocks;
  size_t bytes = 0;
  bt_status alloc(void** p, size_t n);
  void release();
};

}  // namespace bt

// Rounded copies of the factors used by the low-precision solves (same
// row-major block layout as the FP64 arrays; AK / BK are the coupling blocks
// A_{k_s}, B_{k_s} of the interface rows, [S][M][M]).
struct LowFactors {
  float *Dinv = nullptr, *E = nullptr, *G = nullptr, *U = nullptr, *V = nullptr;
  float *AK = nullptr, *BK = nullptr, *R = nullptr, *HL = nullptr, *HR = nullptr;
  bool ready = false;
};

// FP32 transposed copies (element (m, k) at k*M + m) of the interface blocks
// used by the tensor-core path's interface and dichotomy kernels.
struct TransposedF32 {
  float *AK = nullptr, *BK = nullptr, *R = nullptr, *HL = nullptr, *HR = nullptr;
  bool ready = false;
};

// Everything a handle owns.  Block arrays are FP64, row-major M x M blocks.
struct bt_handle_s {
  int device = 0;
  int64_t N = 0, M = 0, S = 0, L = 0;
  int depth = 0;
  int stencil = 0;  // A_j = B_j = I, C_j tridiagonal
  // a stencil whose off-diagonals inside every C_j are exactly -1 and whose
  // diagonal entries lie in [2^-30, 2^30] in magnitude: the refinement forms
  // its residual in FP32 double-word arithmetic (refine.cu, k_resid_dw)
  int stencil_unit = 0;
  int band[4] = {0, 0, 0, 0};  // nonzero diagonals c - r of A_j: [lo, hi]; of B_j: [lo, hi]
  int64_t band_n = 0;          // handles of bt_factor_band: rows n of the band matrix
  double* band_buf = nullptr;  // padded F and X panels of bt_solve_band
  size_t band_bytes = 0;

  bt::DevArena arena;

  // Copies of the operator (A[0] and B[N-1] zeroed): the residual and the
  // adjoint need P after the caller's buffers are gone.
  double* A = nullptr;
  double* B = nullptr;
  double* C = nullptr;

  // Segment factors, indexed by global block row (interface rows unused):
  // D_i^{-1}, E_i = D_i^{-1} A_i, G_i = D_i^{-1} B_i (Gamma), and the coupling
  // responses U_i, V_i of eqs. sub1 / sub2.
  double* Dinv = nullptr;
  double* E = nullptr;
  double* G = nullptr;
  double* U = nullptr;
  double* V = nullptr;
  // Forward responses of the left coupling (Y_a = E_a, Y_i = E_i Y_{i-1}),
  // built on first use (factor_left_responses).
  double* Y = nullptr;

  // Coupling blocks of the interface rows, A_{k_s} and B_{k_s}, [S][M][M].
  double* AK = nullptr;
  double* BK = nullptr;
  // Diagonals of C_j ([N][M][3]: sub, main, super) when the operator is a stencil.
  double* Cdiag = nullptr;
  // The main diagonal of C_j as FP32 pairs [N][M][2]: the rounded value and the
  // rounded remainder (|c - hi - lo| <= 2^-48 |c|).
  float* Cdw = nullptr;

  // Reduced system of eq. red1, [S][M][M].
  double* At = nullptr;
  double* Ct = nullptr;
  double* Bt = nullptr;

  // Dichotomy tree: R[level][j] = block (m, j) of the inverse of the node's
  // sub-matrix for the node containing j at that level; HL / HR indexed by
  // the node's middle unknown m.
  double* R = nullptr;
  double* HL = nullptr;
  double* HR = nullptr;
  std::vector<bt::TreeNode> nodes;     // breadth-first, grouped by level
  std::vector<int> level_off;          // nodes of level l: [level_off[l], level_off[l+1])
  int* d_nodes = nullptr;              // device copy: (l, r, m) per node
  int* d_mid_level = nullptr;          // level at which interface s is the middle unknown

  // Solve scratch (grown on demand): series terms c[level][s] (M x K each).
  double* scratch = nullptr;
  size_t scratch_bytes = 0;

  // Factors of P^T, built on the first adjoint call, and the lambda buffer
  // used when the caller does not ask for dF.
  bt_handle_s* adj = nullptr;
  void* adj_lam = nullptr;
  size_t adj_lam_bytes = 0;

  LowFactors f32;
  TransposedF32 f32t;
  // Tensor-core factor copies [5][N][M][M] (Dinv, E, G, U, V) in BF16 / FP32.
  void* tc_fac_bf16 = nullptr;
  void* tc_fac_tf32 = nullptr;
  void* tc_fac_bf16x3 = nullptr;  // [2][5][N][M][M]: rounded values and their remainders
  // split-BF16 copies [2][4][N][M][M] of Dinv, G, Z = U^T and Y for the
  // forward / backward stage 2 of unit stencils (solve_tc.cu)
  void* tc_fac_fb = nullptr;
  // Split-BF16 copies of the interface blocks for the tensor-core step 2.2,
  // [2][AK (S), BK (S), R (depth*S), HL (S), HR (S)][M][M], and the job table of
  // that step (device; host offsets: F~ jobs, series-term jobs, one group per level).
  void* tc_if_bf16x3 = nullptr;
  void* if_jobs = nullptr;
  std::vector<int> if_off;

  // Refinement buffers (grown on demand): residual panel, work panel,
  // series terms and the device-side refinement state.
  void* lp_r = nullptr;
  void* lp_d = nullptr;
  void* lp_c = nullptr;
  void* lp_x = nullptr;   // FP32 correction panel of the tensor-core solve
  void* lp_x1 = nullptr;  // the first solve's result as an FP32 panel (unit-stencil refinement)
  size_t lp_panel_bytes = 0, lp_d_bytes = 0, lp_c_bytes = 0, lp_x_bytes = 0, lp_x1_bytes = 0;
  void* ir_state = nullptr;
  int lp_gen = 0;  // bumped whenever a refinement buffer is reallocated

  // Exact tensor-core residual (dense blocks, M = 64 or 128): digit slices of
  // the operator rows [3N][7][M][M] (BF16) and their row scales [N][M], built
  // on first use; digit slices of X [7][N][Kp][M] and the per-column maxima
  // and scales [Kp], grown on demand.
  void* dg_fac = nullptr;
  int* dg_ea = nullptr;
  void* dg_x = nullptr;
  size_t dg_x_bytes = 0;
  void* dg_col = nullptr;
  size_t dg_col_bytes = 0;

  // Host-buffer solves (bt_solve_host): two device panel pairs (F, X) of
  // N*M*kc doubles each, their copy streams and events (grown on demand).
  double* hp_buf = nullptr;
  size_t hp_bytes = 0;
  cudaStream_t hp_h2d = nullptr, hp_d2h = nullptr;
  cudaEvent_t hp_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};

  // The refined solve captured as CUDA graphs, one per argument key: a key's
  // second call captures, later calls replay (other calls may come between;
  // the calls on a handle run in order on one stream, so the graphs may share
  // the handle's buffers).  Graphs of buffers that have moved since are
  // dropped; at most kMaxRefineGraphs are kept, least recently used out.
  struct RefineGraph {
    const double* F = nullptr;
    double* X = nullptr;
    int64_t K = 0;
    int precision = -1, max_it = 0, gen = -1, resid = -1;
    double tol = 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;  // last use (handle-local clock)
  };
  static constexpr size_t kMaxRefineGraphs = 64;
  std::vector<RefineGraph> rgraphs;
  uint64_t rg_clock = 0;
  cudaStream_t rg_cap = nullptr;  // private capture streams (the graph, the loop body)
  cudaStream_t rg_cap2 = nullptr;
  bool rg_broken = false;  // a capture failed once: enqueue directly from then on

  bt::Profiler prof;
};

// A batched-solve plan (bt_batch_create): the work-item table of one
// persistent launch over many right-hand-side sets, its scratch, and the CUDA
// graph that replays it.
struct bt_batch_s {
  int device = 0;
  int32_t n = 0;
  int32_t precision = 0;
  bt::DevArena arena;
  void* scratch = nullptr;        // series terms of every set
  void* d_sets = nullptr;         // per-set arguments
  void* d_items = nullptr;        // work items, grouped by stage
  int* d_stage_off = nullptr;     // items of stage t: [off[t], off[t+1])
  int* d_stage_kind = nullptr;
  void* d_ctl = nullptr;          // grid-barrier counters and the status word
  int n_stages = 0;
  int64_t n_items = 0;
  int CW = 4, threads = 0, grid = 0, k_tile = 0;
  size_t smem = 0;
  const void* kernel = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;

  // Refined plans (a precision other than FP64; batch_refined.cu): the sets of
  // each matrix packed into one panel, one refined solve per matrix, all in
  // one CUDA graph.
  struct RGroup {
    bt_handle_s* h = nullptr;
    std::vector<int> members;   // set indices, in packing order
    int nsets = 0, first = 0;   // first: index of its first set in d_norm2
    int64_t K = 0;              // packed columns
    double* F = nullptr;        // packed panels [N][M][K]
    double* X = nullptr;
    void* d_sets = nullptr;     // per-set table
    void* d_blk = nullptr;      // CTAs of the norm launch
    int* d_colset = nullptr;    // set of each packed column
    double* d_colssq = nullptr; // per-column sums of squares of the residual (scratch)
    int64_t nblk = 0;
    int gen = -1;               // the handle's buffer generation when captured
    cudaStream_t q = nullptr;   // the group's branch of the graph
    cudaEvent_t fork = nullptr, join = nullptr;
  };
  bool refined = false;
  bt_opts ropts{};
  std::vector<RGroup> groups;
  std::vector<int> set_group;
  double* d_norm2 = nullptr;    // ||F_s||_F^2 per set
  void* d_state = nullptr;      // each group's refinement state after a run
  int pack_grid = 0;
  cudaStream_t rcap = nullptr;
  std::vector<bt_info> infos;   // per group, filled by bt_batch_status
  bool infos_ready = false;
};

namespace bt {
// Records an event pair around one kernel launch when profiling is on.
struct ProfScope {
  Profiler* p;
  cudaStream_t st;
  ProfScope(bt_handle_s* h, cudaStream_t s, const char* name) : p(h->prof.on ? &h->prof : nullptr), st(s) {
    if (p) {
      Profiler::Rec r{name, p->get(), p->get()};
      cudaEventRecord(r.a, st);
      p->recs.push_back(r);
    }
  }
  ~ProfScope() {
    if (p) cudaEventRecord(p->recs.back().b, st);
  }
};
}  // namespace bt

namespace bt {

// Factorisation (Algorithm 2 stage 1) into an allocated handle.
bt_status factor_f64(bt_handle_s* h, const double* A, const double* B, const double* C,
                     cudaStream_t st);

// FP64 stage-2 pipeline; `stages` in 1..3 (see bt_solve_stages).
bt_status solve_f64(bt_handle_s* h, const double* F, int64_t K, double* X, int stages,
                    cudaStream_t st);

// FP64 stage-2 pipeline with its scratch in the library's fixed array (no allocation).
bt_status solve_f64_noalloc(bt_handle_s* h, const double* F, int64_t K, double* X, cudaStream_t st);

// Grows the handle's scratch pool to at least `bytes`.
bt_status ensure_scratch(bt_handle_s* h, size_t bytes, cudaStream_t st);

// FP32 stage-2 pipeline on the CUDA cores: r -> work panel d (y, W, X~), then
// X = (accumulate ? X : 0) + solution.  Returns at once when *done != 0.
bt_status solve_simt_f32(bt_handle_s* h, const float* r, int64_t K, float* d, float* c, double* X, int accumulate,
                         const int* done, cudaStream_t st);

// Buffers of one tensor-core solve: factor copies, block-transposed residual
// and work panels (leading dimension Kp, a multiple of the column tile), and
// the FP32 series terms [depth][S][M][Kp].
struct TcBuffers {
  const void* fac;
  void* r;
  void* w;
  float* c;
  float* d;  // FP32 correction panel, block-transposed like w
  int64_t Kp;
  // with accumulate 2 and the split-BF16 M = 128 correction: the result as a
  // row-major [N][M][K] FP32 panel here instead of d
  float* drow = nullptr;
};

// Column tile of the tensor-core kernels for a precision and block size (0: unsupported).
int tc_col_tile(int precision, int M);
// Block size of the tensor-core layouts: M padded to 64 or 128 (0 past 128).
// Factor blocks, interface blocks and the block-transposed panels of the
// tensor-core path carry Mt rows (and columns) per block, zero past M.
int tc_M(const bt_handle_s* h);
// Operand planes of a tensor-core precision (2 for the split BF16 precision).
int tc_planes(int precision);
// Builds the tensor-core factor copies for `precision` (once per handle).
bt_status make_tc_factors(bt_handle_s* h, int precision, cudaStream_t st);
// One tensor-core stage-2 solve: r -> w (y, W, X~), then X (+)= solution.
// Y of the handle (see bt_handle_s::Y), built once.
bt_status factor_left_responses(bt_handle_s* h, cudaStream_t st);

// accumulate: 0 X = d (the first solve), 1 X += d, 2 only the FP32 correction
// panel is written (tb.drow when set, else tb.d; X is not touched).
bt_status solve_tc(bt_handle_s* h, int precision, const TcBuffers& tb, int64_t K, double* X, int accumulate,
                   const int* done, int* status, cudaStream_t st);

// Adjoint solve and gradient contractions (bt_solve_adjoint).
bt_status solve_adjoint(bt_handle_s* h, const double* X, const double* G, int64_t K, double* dF, double* dA,
                        double* dB, double* dC, cudaStream_t st);

// Builds h->f32 from the FP64 factors (once per handle).
bt_status make_f32_factors(bt_handle_s* h, cudaStream_t st);

// CTAs of `fn` (threads per CTA, dynamic shared memory) that are resident on
// the whole current device at once: the grid of a grid-stride kernel, so that
// it runs in exactly one wave.
int resident_grid(const void* fn, int threads, size_t smem);

// Batched FP64 solve: builds the item table and launch shape of a plan, and
// enqueues its persistent launch (used directly and under graph capture).
bt_status batch_build(bt_batch_s* b, int32_t n, const bt_handle* hs, const double* const* F, const int64_t* K,
                      double* const* X, const bt_opts& o);
bt_status batch_enqueue(bt_batch_s* b, cudaStream_t st);
// Sets the plan's grid-barrier wait limit (0: the default) and its planted
// failure (a stage index, or -1); synchronous.
bt_status batch_set_debug(bt_batch_s* b, unsigned long long limit_ns, int skip_stage);

// FP64-accurate batched block products on the tensor cores from BF16 digit
// slices (gemm_digits.cu): whether a block size is supported (M = 128), the
// scratch for batches of up to emax entries, and one batched product
// D = alpha X Y + beta Z over a device table of (X, Y, Z, D) pointers per
// entry; *status is set when a bounded wait gave up.
bool digit_gemm_supported(int M);
size_t digit_gemm_bytes(int emax);
bt_status digit_gemm_run(void* scratch, int emax, const double* const* dtab, int E, double alpha, double beta,
                         int* status, cudaStream_t st);

// Refined batches (batch_refined.cu): build (groups, packing tables, prepared
// refinements, the captured graph), run (re-captured first if a handle's
// refinement buffers moved), status (per-group convergence), release.
bt_status rbatch_build(bt_batch_s* b, int32_t n, const bt_handle* hs, const double* const* F, const int64_t* K,
                       double* const* X, const bt_opts& o);
bt_status rbatch_run(bt_batch_s* b, cudaStream_t st);
bt_status rbatch_status(bt_batch_s* b);
void rbatch_release(bt_batch_s* b);

// The FP32 double-word residual (refine.cu) applies: a unit stencil with M % 8 == 0.
bool resid_dw_supported(const bt_handle_s* h);

// Exact residual on the tensor cores (resid_digits.cu): whether it applies to
// the handle for K columns; the digit slices of the operator (once) and the
// scratch for K columns (outside any stream capture); and one residual:
// out_mode 0 -- the tensor-core panel (planes sp, BF16, or FP32 if tr_float,
// leading dimension K rounded up to 128), 1 -- row-major FP32, 2 -- row-major
// FP64; its squared norm is added to rn2[*cur] (rn2[0] if cur is NULL).
// Every kernel returns at once when *done != 0.
bool resid_digits_supported(const bt_handle_s* h, int64_t K);
bt_status resid_digits_prepare(bt_handle_s* h, int64_t K, cudaStream_t st);
bt_status launch_resid_digits(bt_handle_s* h, const double* F, const double* X, int64_t K, int out_mode,
                              bool tr_float, void* out, int sp, const int* done, double* rn2, const int* cur,
                              int* status, cudaStream_t st);

// bt_residual: r = F - P X into R (row-major FP64) by `method` (0 automatic,
// 1 FP64 CUDA cores, 2 tensor-core digits); ||r||_F^2 to *norm2 if non-NULL.
bt_status residual_diag(bt_handle_s* h, const double* F, const double* X, int64_t K, double* R, int method,
                        double* norm2, cudaStream_t st);

// Mixed-precision solve with iterative refinement (bt_solve_ex).  how: 0 run
// (a CUDA graph per argument key, replayed on repeated calls); 1 prepare:
// grow the scratch, build the factor copies, and run the refinement once
// directly on F and X, which builds what the launches build lazily
// (synchronous; no capture may be in progress); 2 record the whole refinement
// into the capture in progress on `rec` (after a `how = 1` call with the same
// K and options; allocates nothing).
// sc (refined batches): the K columns form nsets column sets (colset[c]);
// the refinement then converges when EVERY set s meets
// ||F_s - P X_s||_F <= tol ||F_s||_F, F_s the set's columns scaled by the
// power of two that brings ||F_s||_F into [1/2, 1) (n2[s] = ||F_s||_F^2
// before scaling); colssq: K doubles of zeroed scratch.
struct SetCheck {
  int nsets;
  const int* colset;
  const double* n2;
  double* colssq;
};
bt_status solve_refined(bt_handle_s* h, const double* F, int64_t K, double* X, const bt_opts& o, bt_info* info,
                        int how = 0, cudaStream_t rec = nullptr, const SetCheck* sc = nullptr);
// Bytes of a handle's refinement state, and the bt_info it reports (returns
// the tensor-core status word: non-zero when a bounded wait gave up).
size_t refine_state_bytes();
int refine_state_info(const void* state, bt_info* info);

// Band storage -> block arrays A, B, C of N block rows (band.cu).
bt_status band_to_blocks(const double* ab, int64_t n, int64_t kl, int64_t ku, int64_t N, int64_t M, double* A,
                         double* B, double* C, cudaStream_t st);

}  // namespace bt
