// Refined (mixed-precision) batches: many right-hand-side sets against a few
// factored matrices, as one CUDA graph.
//
// Stage 2 of Algorithm 2 (Section 2.2) is linear in the right-hand side and
// its factors do not depend on it, so all sets of one matrix are columns of
// one panel: the plan packs them side by side, runs ONE refined solve per
// matrix on the packed panel (the factors stream once per matrix instead of
// once per set), and unpacks the columns into each set's X.  The matrices'
// panels run on concurrent branches of the graph; every refinement loop is a
// device-side WHILE node, so a run is one graph launch with no host work.
//
// Accuracy per set.  Before packing, set s is scaled by 2^-e_s with
// 2^(e_s - 1) <= ||F_s||_F < 2^e_s (exact in binary floating point: every
// packed set has 1/2 <= ||F'_s||_F < 1 whatever its magnitude, and
// X_s = 2^e_s X'_s exactly).  The packed refinement stops when every set's own
// residual meets ||R'_s||_F <= tol ||F'_s||_F (SetCheck: the sets' sums of
// squares of the residual panel after each pass), the relative residual a
// solve of that set alone would be held to.
#include "bt_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace bt {
namespace {

constexpr int64_t kNormChunk = 1 << 15;  // entries of one set per CTA of the norm launch
constexpr int kMaxPackSets = 1024;       // sets of one matrix (the pack kernels' shared tables)

struct PackSet {
  const double* F;
  double* X;
  int64_t K;   // columns of the set
  int64_t c0;  // first column in the packed panel
};
struct NormBlk {
  int32_t set;
  int32_t pad;
  int64_t off;  // first entry of the set's [N][M][K] array
};

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  v = 0.0;
  if (threadIdx.x < 32) {
    v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// ||F_s||_F^2 of every set: CTA b sums the chunk blk[b] of one set.
__global__ void __launch_bounds__(256) k_set_norm2(const PackSet* __restrict__ sets, const NormBlk* __restrict__ blk,
                                                   int64_t rows, double* __restrict__ norm2) {
  const NormBlk b = blk[blockIdx.x];
  const PackSet p = sets[b.set];
  const int64_t end = min(b.off + kNormChunk, rows * p.K);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int64_t i = b.off + threadIdx.x;
  for (; i + 768 < end; i += 1024) {
    const double v0 = __ldg(p.F + i), v1 = __ldg(p.F + i + 256), v2 = __ldg(p.F + i + 512), v3 = __ldg(p.F + i + 768);
    a0 = fma(v0, v0, a0);
    a1 = fma(v1, v1, a1);
    a2 = fma(v2, v2, a2);
    a3 = fma(v3, v3, a3);
  }
  for (; i < end; i += 256) {
    const double v = __ldg(p.F + i);
    a0 = fma(v, v, a0);
  }
  const double s = block_sum((a0 + a1) + (a2 + a3));
  if (threadIdx.x == 0) atomicAdd(norm2 + b.set, s);
}

// The exponent e with 2^(e-1) <= sqrt(n2) < 2^e (0 for a zero or non-finite norm).
__device__ __forceinline__ int set_exponent(double n2) {
  if (!(n2 > 0.0) || !(n2 < INFINITY)) return 0;
  int e = 0;
  frexp(sqrt(n2), &e);
  return e;
}

// dir 0: Fp[r][c0_s + c] = 2^-e_s F_s[r][c]; dir 1: X_s[r][c] = 2^e_s Xp[r][c0_s + c].
// CTAs take the N*M block-row entries r in turn; the threads sweep the packed
// columns of a row, four loads in flight each, the set of a packed column
// from colset: coalesced on the packed side and within each set.
constexpr int kPackU = 4;
__global__ void __launch_bounds__(256) k_pack_sets(const PackSet* __restrict__ sets, int nsets,
                                                   const int* __restrict__ colset, const double* __restrict__ norm2,
                                                   int64_t rows, int64_t Kt, double* __restrict__ P, int dir) {
  __shared__ PackSet ts[kMaxPackSets];
  __shared__ double sc[kMaxPackSets];
  for (int s = threadIdx.x; s < nsets; s += blockDim.x) {
    ts[s] = sets[s];
    const int e = set_exponent(norm2[s]);
    sc[s] = ldexp(1.0, dir == 0 ? -e : e);
  }
  __syncthreads();
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    double* pr = P + r * Kt;
    for (int64_t cb = 0; cb < Kt; cb += (int64_t)kPackU * blockDim.x) {
      double v[kPackU];
      int si[kPackU];
#pragma unroll
      for (int u = 0; u < kPackU; ++u) {
        const int64_t c = cb + threadIdx.x + (int64_t)u * blockDim.x;
        si[u] = c < Kt ? __ldg(colset + c) : -1;
        if (si[u] >= 0) {
          const PackSet& p = ts[si[u]];
          v[u] = dir == 0 ? __ldg(p.F + r * p.K + (c - p.c0)) : pr[c];
        }
      }
#pragma unroll
      for (int u = 0; u < kPackU; ++u) {
        if (si[u] < 0) continue;
        const int64_t c = cb + threadIdx.x + (int64_t)u * blockDim.x;
        const PackSet& p = ts[si[u]];
        if (dir == 0)
          pr[c] = v[u] * sc[si[u]];
        else
          p.X[r * p.K + (c - p.c0)] = v[u] * sc[si[u]];
      }
    }
  }
}

bt_status record_plan(bt_batch_s* b);

// Prepares every matrix's refinement for its packed width (allocations,
// factor copies, one direct run on the packed panel) and captures the plan's
// graph.
bt_status prepare_and_capture(bt_batch_s* b) {
  for (auto& g : b->groups) {
    bt_opts o = b->ropts;
    o.stream = nullptr;
    const SetCheck sc{g.nsets, g.d_colset, b->d_norm2 + g.first, g.d_colssq};
    BT_TRY(solve_refined(g.h, g.F, g.K, g.X, o, nullptr, 1, nullptr, &sc));
    BT_CUDA(cudaDeviceSynchronize());
  }
  return record_plan(b);
}

bt_status record_plan(bt_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  if (!b->rcap) BT_CUDA(cudaStreamCreateWithFlags(&b->rcap, cudaStreamNonBlocking));
  for (auto& g : b->groups) {
    if (!g.q) BT_CUDA(cudaStreamCreateWithFlags(&g.q, cudaStreamNonBlocking));
    if (!g.fork) BT_CUDA(cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming));
    if (!g.join) BT_CUDA(cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming));
  }
  const size_t sb = refine_state_bytes();
  cudaStream_t cs = b->rcap;
  BT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  bt_status st = BT_OK;
  auto fail = [&](bt_status s) {
    if (st == BT_OK) st = s;
  };
  if (cudaMemsetAsync(b->d_norm2, 0, sizeof(double) * b->n, cs) != cudaSuccess) fail(BT_ERR_CUDA);
  for (size_t gi = 0; gi < b->groups.size() && st == BT_OK; ++gi) {
    auto& g = b->groups[gi];
    const int64_t rows = g.h->N * g.h->M;
    double* n2 = b->d_norm2 + g.first;
    const PackSet* sets = reinterpret_cast<const PackSet*>(g.d_sets);
    const bool prof = g.h->prof.on;
    g.h->prof.on = false;  // no event records inside the graph
    if (cudaEventRecord(g.fork, cs) != cudaSuccess || cudaStreamWaitEvent(g.q, g.fork, 0) != cudaSuccess) {
      fail(BT_ERR_CUDA);
    } else {
      k_set_norm2<<<(unsigned)g.nblk, 256, 0, g.q>>>(sets, reinterpret_cast<const NormBlk*>(g.d_blk), rows, n2);
      const unsigned grid = (unsigned)std::min<int64_t>(rows, b->pack_grid);
      k_pack_sets<<<grid, 256, 0, g.q>>>(sets, g.nsets, g.d_colset, n2, rows, g.K, g.F, 0);
      bt_opts o = b->ropts;
      o.stream = g.q;
      const SetCheck sc{g.nsets, g.d_colset, n2, g.d_colssq};
      if (cudaMemsetAsync(g.d_colssq, 0, sizeof(double) * g.K, g.q) != cudaSuccess) fail(BT_ERR_CUDA);
      fail(solve_refined(g.h, g.F, g.K, g.X, o, nullptr, 2, g.q, &sc));
      k_pack_sets<<<grid, 256, 0, g.q>>>(sets, g.nsets, g.d_colset, n2, rows, g.K, g.X, 1);
      if (cudaMemcpyAsync(static_cast<char*>(b->d_state) + gi * sb, g.h->ir_state, sb, cudaMemcpyDeviceToDevice,
                          g.q) != cudaSuccess ||
          cudaEventRecord(g.join, g.q) != cudaSuccess || cudaStreamWaitEvent(cs, g.join, 0) != cudaSuccess)
        fail(BT_ERR_CUDA);
    }
    g.h->prof.on = prof;
  }
  if (cudaGetLastError() != cudaSuccess) fail(BT_ERR_CUDA);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (st == BT_OK && (e != cudaSuccess || !graph)) {
    set_error(std::string("bt_batch_create: capturing the refined batch failed: ") + cudaGetErrorString(e));
    st = BT_ERR_CUDA;
  }
  if (st == BT_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
    set_error("bt_batch_create: instantiating the refined batch's graph failed");
    st = BT_ERR_CUDA;
  }
  if (st != BT_OK) {
    if (graph) cudaGraphDestroy(graph);
    b->exec = nullptr;
    cudaGetLastError();
    return st;
  }
  b->graph = graph;
  for (auto& g : b->groups) g.gen = g.h->lp_gen;
  return BT_OK;
}

}  // namespace

bt_status rbatch_build(bt_batch_s* b, int32_t n, const bt_handle* hs, const double* const* F, const int64_t* K,
                       double* const* X, const bt_opts& o) {
  b->refined = true;
  b->ropts = o;
  b->ropts.stream = nullptr;
  if (!(b->ropts.tol > 0)) b->ropts.tol = 1e-10;
  // sets grouped by matrix, in the order the matrices first appear
  for (int32_t i = 0; i < n; ++i) {
    size_t gi = 0;
    while (gi < b->groups.size() && b->groups[gi].h != hs[i]) ++gi;
    if (gi == b->groups.size()) {
      bt_batch_s::RGroup g;
      g.h = hs[i];
      b->groups.push_back(g);
    }
    b->groups[gi].members.push_back(i);
  }
  b->set_group.assign((size_t)n, 0);
  BT_TRY(b->arena.alloc((void**)&b->d_norm2, sizeof(double) * (size_t)n));
  BT_TRY(b->arena.alloc(&b->d_state, refine_state_bytes() * b->groups.size()));
  int first = 0;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    auto& g = b->groups[gi];
    g.nsets = (int)g.members.size();
    if (g.nsets > kMaxPackSets) {
      set_error("bt_batch_create: at most " + std::to_string(kMaxPackSets) + " sets per matrix in a refined batch");
      return BT_ERR_ARG;
    }
    g.first = first;
    first += g.nsets;
    const int64_t rows = g.h->N * g.h->M;
    std::vector<PackSet> ps;
    std::vector<NormBlk> nb;
    std::vector<int> cs;
    int64_t c0 = 0;
    for (int k = 0; k < g.nsets; ++k) {
      const int i = g.members[k];
      b->set_group[(size_t)i] = (int)gi;
      ps.push_back(PackSet{F[i], X[i], K[i], c0});
      for (int64_t off = 0; off < rows * K[i]; off += kNormChunk) nb.push_back(NormBlk{k, 0, off});
      cs.insert(cs.end(), (size_t)K[i], k);
      c0 += K[i];
    }
    g.K = c0;
    g.nblk = (int64_t)nb.size();
    const size_t panel = (size_t)rows * g.K * sizeof(double);
    BT_TRY(b->arena.alloc((void**)&g.F, panel));
    BT_TRY(b->arena.alloc((void**)&g.X, panel));
    BT_TRY(b->arena.alloc(&g.d_sets, ps.size() * sizeof(PackSet)));
    BT_TRY(b->arena.alloc(&g.d_blk, nb.size() * sizeof(NormBlk)));
    BT_TRY(b->arena.alloc((void**)&g.d_colset, cs.size() * sizeof(int)));
    BT_TRY(b->arena.alloc((void**)&g.d_colssq, cs.size() * sizeof(double)));
    BT_CUDA(cudaMemset(g.d_colssq, 0, cs.size() * sizeof(double)));
    BT_CUDA(cudaMemcpy(g.d_colset, cs.data(), cs.size() * sizeof(int), cudaMemcpyHostToDevice));
    BT_CUDA(cudaMemset(g.F, 0, panel));  // the preparing run solves zeros
    BT_CUDA(cudaMemcpy(g.d_sets, ps.data(), ps.size() * sizeof(PackSet), cudaMemcpyHostToDevice));
    BT_CUDA(cudaMemcpy(g.d_blk, nb.data(), nb.size() * sizeof(NormBlk), cudaMemcpyHostToDevice));
  }
  b->pack_grid = resident_grid(reinterpret_cast<const void*>(&k_pack_sets), 256, 0);
  return prepare_and_capture(b);
}

bt_status rbatch_run(bt_batch_s* b, cudaStream_t st) {
  bool moved = false;  // a handle's refinement buffers were reallocated by another call
  for (auto& g : b->groups) moved = moved || g.gen != g.h->lp_gen;
  if (moved || !b->exec) BT_TRY(prepare_and_capture(b));
  BT_CUDA(cudaGraphLaunch(b->exec, st));
  return BT_OK;
}

bt_status rbatch_status(bt_batch_s* b) {
  const size_t sb = refine_state_bytes();
  std::vector<char> hs(sb * b->groups.size());
  BT_CUDA(cudaMemcpy(hs.data(), b->d_state, hs.size(), cudaMemcpyDeviceToHost));
  b->infos.assign(b->groups.size(), bt_info{});
  bt_status worst = BT_OK;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const int ks = refine_state_info(hs.data() + gi * sb, &b->infos[gi]);
    if (ks != 0) {
      set_error("bt_batch: a tensor-core kernel gave up a bounded wait (code " + std::to_string(ks) + ")");
      worst = BT_ERR_TIMEOUT;
    } else if (!b->infos[gi].converged && worst == BT_OK) {
      set_error("bt_batch: the refinement of matrix group " + std::to_string(gi) +
                " stopped at relative residual " + std::to_string(b->infos[gi].rel_res));
      worst = BT_ERR_NOCONV;
    }
  }
  b->infos_ready = true;
  return worst;
}

void rbatch_release(bt_batch_s* b) {
  for (auto& g : b->groups) {
    if (g.q) cudaStreamDestroy(g.q);
    if (g.fork) cudaEventDestroy(g.fork);
    if (g.join) cudaEventDestroy(g.join);
    g.q = nullptr;
    g.fork = g.join = nullptr;
  }
  if (b->rcap) cudaStreamDestroy(b->rcap);
  b->rcap = nullptr;
}

}  // namespace bt
