// C-ABI entry points: argument validation, handle lifetime, dispatch.
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>

#include "bt_internal.cuh"

namespace bt {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

bt_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? BT_ERR_OOM : BT_ERR_CUDA;
}

int resident_grid(const void* fn, int threads, size_t smem) {
  // cached per (device, kernel, shape): the first query of a kernel may load
  // its module, which must not happen inside a stream capture
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  const auto key = std::make_tuple(dev, fn, threads, smem);
  {
    std::lock_guard<std::mutex> g(mu);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 152;
  }
  std::lock_guard<std::mutex> g(mu);
  cache[key] = sms * per_sm;
  return sms * per_sm;
}

bt_status DevArena::alloc(void** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 16;
  cudaError_t e = cudaMalloc(p, n);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error(std::string("device allocation of ") + std::to_string(n) + " bytes failed: " + cudaGetErrorString(e));
    return BT_ERR_OOM;
  }
  blocks.push_back(*p);
  bytes += n;
  return BT_OK;
}

void DevArena::release() {
  for (void* p : blocks) cudaFree(p);
  blocks.clear();
  bytes = 0;
}

cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Profiler::collect() {
  for (const Rec& r : recs) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    size_t k = 0;
    while (k < names.size() && names[k] != r.name) ++k;
    if (k == names.size()) {
      names.push_back(r.name);
      launches.push_back(0);
      total_ms.push_back(0.0);
    }
    launches[k] += 1;
    total_ms[k] += ms;
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  recs.clear();
}

void Profiler::destroy() {
  for (const Rec& r : recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  recs.clear();
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
  pool.clear();
}

static void destroy_handle(bt_handle_s* h) {
  if (!h) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  if (h->adj) destroy_handle(h->adj);
  h->prof.destroy();
  h->arena.release();
  if (h->scratch) cudaFree(h->scratch);
  for (void* q : {h->lp_r, h->lp_d, h->lp_c, h->lp_x, h->lp_x1, h->ir_state, h->adj_lam, h->dg_fac,
                  static_cast<void*>(h->dg_ea), h->dg_x, h->dg_col})
    if (q) cudaFree(q);
  for (auto& g : h->rgraphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  if (h->hp_buf) cudaFree(h->hp_buf);
  if (h->band_buf) cudaFree(h->band_buf);
  if (h->hp_h2d) cudaStreamDestroy(h->hp_h2d);
  if (h->hp_d2h) cudaStreamDestroy(h->hp_d2h);
  for (cudaEvent_t e : h->hp_ev)
    if (e) cudaEventDestroy(e);
  if (h->rg_cap) cudaStreamDestroy(h->rg_cap);
  if (h->rg_cap2) cudaStreamDestroy(h->rg_cap2);
  cudaSetDevice(prev);
  delete h;
}

static bt_status check_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  if (prop.major != 10 || prop.minor != 3) {
    set_error("this library is built for sm_103a (GB300); the current device is sm_" +
              std::to_string(prop.major) + std::to_string(prop.minor));
    return BT_ERR_CUDA;
  }
  return BT_OK;
}

bt_status make_handle(int64_t N, int64_t M, const double* A, const double* B, const double* C, int64_t S,
                      cudaStream_t st, bt_handle_s** out) {
  *out = nullptr;
  bt_handle_s* h = new (std::nothrow) bt_handle_s();
  if (!h) {
    set_error("bt_factor: host allocation failed");
    return BT_ERR_OOM;
  }
  cudaGetDevice(&h->device);
  h->N = N;
  h->M = M;
  h->S = S;
  h->L = N / S;
  bt_status s = factor_f64(h, A, B, C, st);
  if (s != BT_OK) {
    destroy_handle(h);
    return s;
  }
  *out = h;
  return BT_OK;
}

}  // namespace bt

using namespace bt;

extern "C" {

const char* bt_strerror(bt_status s) {
  switch (s) {
    case BT_OK: return "ok";
    case BT_ERR_ARG: return "invalid argument";
    case BT_ERR_SINGULAR: return "singular or non-finite pivot block";
    case BT_ERR_CUDA: return "CUDA error";
    case BT_ERR_NOCONV: return "iterative refinement did not converge";
    case BT_ERR_TIMEOUT: return "device-side wait timed out";
    case BT_ERR_OOM: return "out of device memory";
    case BT_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

const char* bt_last_error(void) { return g_last_error.c_str(); }

bt_status bt_factor(int64_t N, int64_t M, const double* A, const double* B, const double* C, int64_t S,
                    void* stream, bt_handle* out) {
  if (!out) {
    set_error("bt_factor: out is NULL");
    return BT_ERR_ARG;
  }
  *out = nullptr;
  if (N < 1 || M < 1 || M > 1024 || S < 1 || S > N || N % S != 0) {
    set_error("bt_factor: need N >= 1, 1 <= M <= 1024, 1 <= S <= N and N % S == 0");
    return BT_ERR_ARG;
  }
  if (!A || !B || !C) {
    set_error("bt_factor: A, B and C must be device pointers");
    return BT_ERR_ARG;
  }
  BT_TRY(check_device());
  return make_handle(N, M, A, B, C, S, (cudaStream_t)stream, out);
}

bt_status bt_factor_band(int64_t n, int64_t kl, int64_t ku, const double* ab, int64_t M, int64_t S, void* stream,
                         bt_handle* out) {
  if (!out) {
    set_error("bt_factor_band: out is NULL");
    return BT_ERR_ARG;
  }
  *out = nullptr;
  if (n < 1 || M < 1 || M > 1024 || kl < 0 || ku < 0 || kl > M || ku > M || S < 1 || S > (n + M - 1) / M) {
    set_error("bt_factor_band: need n >= 1, 1 <= M <= 1024, 0 <= kl, ku <= M and 1 <= S <= ceil(n / M)");
    return BT_ERR_ARG;
  }
  if (!ab) {
    set_error("bt_factor_band: ab must be a device pointer");
    return BT_ERR_ARG;
  }
  BT_TRY(check_device());
  const cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = ((n + M - 1) / M + S - 1) / S * S;
  const size_t bytes = (size_t)N * M * M * sizeof(double);
  double* blocks = nullptr;
  BT_CUDA(cudaMallocAsync((void**)&blocks, 3 * bytes, st));
  double *A = blocks, *B = blocks + (size_t)N * M * M, *C = blocks + 2 * (size_t)N * M * M;
  bt_status s = band_to_blocks(ab, n, kl, ku, N, M, A, B, C, st);
  if (s == BT_OK) s = make_handle(N, M, A, B, C, S, st, out);
  // make_handle has synchronised the stream (or failed): the blocks are free to go
  const cudaError_t e = cudaFreeAsync(blocks, st);
  if (s != BT_OK) return s;
  if (e != cudaSuccess) {
    bt_destroy(*out);
    *out = nullptr;
    return cuda_fail(e, "cudaFreeAsync");
  }
  (*out)->band_n = n;
  return BT_OK;
}

bt_status bt_solve_band(bt_handle h, const double* F, int64_t K, double* X, const bt_opts* opts, bt_info* info) {
  if (!h || !F || !X || K < 1 || h->band_n < 1) {
    set_error("bt_solve_band: need a handle of bt_factor_band, device F and X, K >= 1");
    return BT_ERR_ARG;
  }
  const int64_t n = h->band_n, NM = h->N * h->M;
  if (n == NM) return bt_solve_ex(h, F, K, X, opts, info);
  const size_t bytes = (size_t)n * K * sizeof(double);
  const char* f0 = reinterpret_cast<const char*>(F);
  const char* x0 = reinterpret_cast<const char*>(X);
  if (f0 < x0 + bytes && x0 < f0 + bytes) {
    set_error("bt_solve_band: X must not overlap F");
    return BT_ERR_ARG;
  }
  const cudaStream_t st = (cudaStream_t)(opts ? opts->stream : nullptr);
  const size_t panel = (size_t)NM * K * sizeof(double);
  if (2 * panel > h->band_bytes) {
    BT_CUDA(cudaDeviceSynchronize());
    if (h->band_buf) BT_CUDA(cudaFree(h->band_buf));
    h->band_buf = nullptr;
    h->band_bytes = 0;
    const cudaError_t e = cudaMalloc((void**)&h->band_buf, 2 * panel);
    if (e != cudaSuccess) {
      h->band_buf = nullptr;
      set_error(std::string("bt_solve_band: panel allocation failed: ") + cudaGetErrorString(e));
      return BT_ERR_OOM;
    }
    h->band_bytes = 2 * panel;
  }
  // rows n .. N*M-1 of the padded system are identity rows with zero right-hand side
  double* Fp = h->band_buf;
  double* Xp = h->band_buf + (size_t)NM * K;
  BT_CUDA(cudaMemcpyAsync(Fp, F, bytes, cudaMemcpyDeviceToDevice, st));
  BT_CUDA(cudaMemsetAsync(Fp + (size_t)n * K, 0, panel - bytes, st));
  const bt_status s = bt_solve_ex(h, Fp, K, Xp, opts, info);
  if (s != BT_OK && s != BT_ERR_NOCONV) return s;  // NOCONV still leaves the last iterate
  BT_CUDA(cudaMemcpyAsync(X, Xp, bytes, cudaMemcpyDeviceToDevice, st));
  return s;
}

bt_status bt_solve_stages(bt_handle h, const double* F, int64_t K, double* X, int32_t stages, void* stream) {
  if (!h || !F || !X || K < 1 || stages < 1 || stages > 3) {
    set_error("bt_solve: need a handle, device F and X, K >= 1 (stages in 1..3)");
    return BT_ERR_ARG;
  }
  const size_t bytes = (size_t)h->N * h->M * K * sizeof(double);
  const char* f0 = reinterpret_cast<const char*>(F);
  const char* x0 = reinterpret_cast<const char*>(X);
  if (f0 < x0 + bytes && x0 < f0 + bytes) {
    set_error("bt_solve: X must not overlap F");
    return BT_ERR_ARG;
  }
  return solve_f64(h, F, K, X, stages, (cudaStream_t)stream);
}

bt_status bt_solve_noalloc(bt_handle h, const double* F, int64_t K, double* X, void* stream) {
  if (!h || !F || !X || K < 1) {
    set_error("bt_solve_noalloc: need a handle, device F and X, K >= 1");
    return BT_ERR_ARG;
  }
  if ((uint64_t)K > (uint64_t)INT64_MAX / ((uint64_t)h->N * h->M * sizeof(double))) {
    set_error("bt_solve_noalloc: K too large for the scratch array");
    return BT_ERR_ARG;
  }
  const size_t bytes = (size_t)h->N * h->M * K * sizeof(double);
  const char* f0 = reinterpret_cast<const char*>(F);
  const char* x0 = reinterpret_cast<const char*>(X);
  if (f0 < x0 + bytes && x0 < f0 + bytes) {
    set_error("bt_solve_noalloc: X must not overlap F");
    return BT_ERR_ARG;
  }
  return solve_f64_noalloc(h, F, K, X, (cudaStream_t)stream);
}

bt_status bt_solve_host(bt_handle h, const double* F, int64_t K, double* X, const bt_opts* opts) {
  if (!h || !F || !X || K < 1) {
    set_error("bt_solve_host: need a handle, host F and X, K >= 1");
    return BT_ERR_ARG;
  }
  bt_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  const cudaStream_t cs = (cudaStream_t)o.stream;
  const int64_t NM = h->N * h->M;
  // column chunks: the tensor-core tile (128), at least about four chunks per call
  const int64_t KC = K <= 128 ? K : std::max<int64_t>(128, ((K + 3) / 4 + 127) / 128 * 128);
  const size_t panel = (size_t)NM * KC * sizeof(double);
  if (4 * panel > h->hp_bytes) {
    BT_CUDA(cudaDeviceSynchronize());
    if (h->hp_buf) BT_CUDA(cudaFree(h->hp_buf));
    h->hp_buf = nullptr;
    h->hp_bytes = 0;
    const cudaError_t e = cudaMalloc((void**)&h->hp_buf, 4 * panel);
    if (e != cudaSuccess) {
      h->hp_buf = nullptr;
      set_error(std::string("bt_solve_host: panel allocation failed: ") + cudaGetErrorString(e));
      return BT_ERR_OOM;
    }
    h->hp_bytes = 4 * panel;
  }
  if (!h->hp_h2d) BT_CUDA(cudaStreamCreateWithFlags(&h->hp_h2d, cudaStreamNonBlocking));
  if (!h->hp_d2h) BT_CUDA(cudaStreamCreateWithFlags(&h->hp_d2h, cudaStreamNonBlocking));
  for (cudaEvent_t& e : h->hp_ev)
    if (!e) BT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaEvent_t* ev_in = h->hp_ev;       // chunk uploaded into pair b
  cudaEvent_t* ev_sol = h->hp_ev + 2;  // chunk solved
  cudaEvent_t* ev_out = h->hp_ev + 4;  // chunk downloaded: pair b free again
  // the inputs may have been written on the compute stream
  BT_CUDA(cudaEventRecord(ev_sol[0], cs));
  BT_CUDA(cudaStreamWaitEvent(h->hp_h2d, ev_sol[0], 0));
  const size_t pitch = (size_t)K * sizeof(double);
  const int64_t nch = (K + KC - 1) / KC;
  for (int64_t c = 0; c < nch; ++c) {
    const int b = (int)(c & 1);
    const int64_t c0 = c * KC, kc = std::min<int64_t>(KC, K - c0);
    double* Fd = h->hp_buf + (size_t)(2 * b) * NM * KC;
    double* Xd = h->hp_buf + (size_t)(2 * b + 1) * NM * KC;
    const size_t w = (size_t)kc * sizeof(double);
    if (c >= 2) BT_CUDA(cudaStreamWaitEvent(h->hp_h2d, ev_out[b], 0));
    BT_CUDA(cudaMemcpy2DAsync(Fd, w, F + c0, pitch, w, (size_t)NM, cudaMemcpyHostToDevice, h->hp_h2d));
    BT_CUDA(cudaEventRecord(ev_in[b], h->hp_h2d));
    BT_CUDA(cudaStreamWaitEvent(cs, ev_in[b], 0));
    BT_TRY(bt_solve_ex(h, Fd, kc, Xd, &o, nullptr));
    BT_CUDA(cudaEventRecord(ev_sol[b], cs));
    BT_CUDA(cudaStreamWaitEvent(h->hp_d2h, ev_sol[b], 0));
    BT_CUDA(cudaMemcpy2DAsync(X + c0, pitch, Xd, w, w, (size_t)NM, cudaMemcpyDeviceToHost, h->hp_d2h));
    BT_CUDA(cudaEventRecord(ev_out[b], h->hp_d2h));
  }
  BT_CUDA(cudaStreamSynchronize(h->hp_d2h));
  BT_CUDA(cudaStreamSynchronize(cs));
  return BT_OK;
}

bt_status bt_solve(bt_handle h, const double* F, int64_t K, double* X, void* stream) {
  return bt_solve_stages(h, F, K, X, 3, stream);
}

bt_status bt_solve_ex(bt_handle h, const double* F, int64_t K, double* X, const bt_opts* opts, bt_info* info) {
  bt_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.precision == BT_PREC_F64) {
    BT_TRY(bt_solve_stages(h, F, K, X, 3, o.stream));
    if (info) {
      BT_CUDA(cudaStreamSynchronize((cudaStream_t)o.stream));
      info->iters = 0;
      info->converged = 1;
      info->rel_res = -1.0;
      info->rel_res0 = -1.0;
    }
    return BT_OK;
  }
  if (!h || !F || !X || K < 1) {
    set_error("bt_solve_ex: need a handle, device F and X, K >= 1");
    return BT_ERR_ARG;
  }
  if (o.precision < 0 || o.precision > 4) {
    set_error("bt_solve_ex: unknown precision");
    return BT_ERR_ARG;
  }
  if (o.residual < 0 || o.residual > 3) {
    set_error("bt_solve_ex: unknown residual method");
    return BT_ERR_ARG;
  }
  const size_t bytes = (size_t)h->N * h->M * K * sizeof(double);
  const char* f0 = reinterpret_cast<const char*>(F);
  const char* x0 = reinterpret_cast<const char*>(X);
  if (f0 < x0 + bytes && x0 < f0 + bytes) {
    set_error("bt_solve_ex: X must not overlap F");
    return BT_ERR_ARG;
  }
  return solve_refined(h, F, K, X, o, info);
}

bt_status bt_residual(bt_handle h, const double* F, const double* X, int64_t K, double* R, int32_t method,
                      double* norm2, void* stream) {
  if (!h || !F || !X || !R || K < 1) {
    set_error("bt_residual: need a handle, device F, X and R, K >= 1");
    return BT_ERR_ARG;
  }
  if (method < 0 || method > 3) {
    set_error("bt_residual: unknown method");
    return BT_ERR_ARG;
  }
  const size_t bytes = (size_t)h->N * h->M * K * sizeof(double);
  const char* r0 = reinterpret_cast<const char*>(R);
  for (const double* p : {F, X}) {
    const char* q = reinterpret_cast<const char*>(p);
    if (r0 < q + bytes && q < r0 + bytes) {
      set_error("bt_residual: R must not overlap F or X");
      return BT_ERR_ARG;
    }
  }
  return residual_diag(h, F, X, K, R, method, norm2, (cudaStream_t)stream);
}

bt_status bt_solve_adjoint(bt_handle h, const double* X, const double* G, int64_t K, double* dF, double* dA,
                           double* dB, double* dC, void* stream) {
  if (!h || !X || !G || K < 1) {
    set_error("bt_solve_adjoint: need a handle, device X and G, K >= 1");
    return BT_ERR_ARG;
  }
  if (h->N > 65535) {
    set_error("bt_solve_adjoint: N > 65535 is not supported");
    return BT_ERR_UNSUPPORTED;
  }
  const size_t bytes = (size_t)h->N * h->M * K * sizeof(double);
  if (dF) {
    const char* g0 = reinterpret_cast<const char*>(G);
    const char* f0 = reinterpret_cast<const char*>(dF);
    if (g0 < f0 + bytes && f0 < g0 + bytes) {
      set_error("bt_solve_adjoint: dF must not overlap G");
      return BT_ERR_ARG;
    }
  }
  return solve_adjoint(h, X, G, K, dF, dA, dB, dC, (cudaStream_t)stream);
}

void bt_destroy(bt_handle h) { destroy_handle(h); }

// ---------------------------------------------------------------- batches
static void destroy_batch(bt_batch_s* b) {
  if (!b) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  rbatch_release(b);
  b->arena.release();
  cudaSetDevice(prev);
  delete b;
}

static bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + nb && y < x + na;
}

bt_status bt_batch_create(int32_t n, const bt_handle* h, const double* const* F, const int64_t* K,
                          double* const* X, const bt_opts* opts, bt_batch* out) {
  if (!out) {
    set_error("bt_batch_create: out is NULL");
    return BT_ERR_ARG;
  }
  *out = nullptr;
  if (n < 1 || !h || !F || !K || !X) {
    set_error("bt_batch_create: need n >= 1 and host arrays h, F, K, X");
    return BT_ERR_ARG;
  }
  bt_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.precision < 0 || o.precision > 4) {
    set_error("bt_batch_create: unknown precision");
    return BT_ERR_ARG;
  }
  if (o.residual < 0 || o.residual > 3) {
    set_error("bt_batch_create: unknown residual method");
    return BT_ERR_ARG;
  }
  if (o.k_tile < 0) {
    set_error("bt_batch_create: k_tile must be >= 0");
    return BT_ERR_ARG;
  }
  int dev = 0;
  BT_CUDA(cudaGetDevice(&dev));
  for (int32_t i = 0; i < n; ++i) {
    if (!h[i] || !F[i] || !X[i] || K[i] < 1) {
      set_error("bt_batch_create: set " + std::to_string(i) + " needs a handle, device F and X, K >= 1");
      return BT_ERR_ARG;
    }
    if (h[i]->device != dev || h[i]->M != h[0]->M) {
      set_error("bt_batch_create: every handle must be on the current device and share one block size M");
      return BT_ERR_ARG;
    }
  }
  for (int32_t i = 0; i < n; ++i) {
    const size_t bi = (size_t)h[i]->N * h[i]->M * K[i] * sizeof(double);
    for (int32_t j = 0; j < n; ++j) {
      const size_t bj = (size_t)h[j]->N * h[j]->M * K[j] * sizeof(double);
      if (overlaps(X[i], bi, F[j], bj) || (j != i && overlaps(X[i], bi, X[j], bj))) {
        set_error("bt_batch_create: X of set " + std::to_string(i) + " overlaps the panels of set " +
                  std::to_string(j));
        return BT_ERR_ARG;
      }
    }
  }
  bt_batch_s* b = new (std::nothrow) bt_batch_s();
  if (!b) {
    set_error("bt_batch_create: host allocation failed");
    return BT_ERR_OOM;
  }
  b->device = dev;
  b->n = n;
  b->precision = o.precision;
  if (o.precision != BT_PREC_F64) {
    const bt_status rs = rbatch_build(b, n, h, F, K, X, o);
    if (rs != BT_OK) {
      destroy_batch(b);
      return rs;
    }
    *out = b;
    return BT_OK;
  }
  bt_status st = batch_build(b, n, h, F, K, X, o);
  if (st == BT_OK) {
    // capture one run into a CUDA graph on a private stream
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const bt_status q = batch_enqueue(b, cs);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (q == BT_OK && e == cudaSuccess && g) {
          if (cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess)
            b->graph = g;
          else
            cudaGraphDestroy(g);
        } else if (g) {
          cudaGraphDestroy(g);
        }
      }
      cudaStreamDestroy(cs);
    }
    cudaGetLastError();  // a failed capture leaves plain launches in use
  }
  if (st != BT_OK) {
    destroy_batch(b);
    return st;
  }
  *out = b;
  return BT_OK;
}

bt_status bt_batch_run(bt_batch b, void* stream) {
  if (!b) {
    set_error("bt_batch_run: NULL plan");
    return BT_ERR_ARG;
  }
  if (b->refined) return rbatch_run(b, (cudaStream_t)stream);
  if (b->exec) {
    BT_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return BT_OK;
  }
  return batch_enqueue(b, (cudaStream_t)stream);
}

bt_status bt_batch_status(bt_batch b) {
  if (!b) {
    set_error("bt_batch_status: NULL plan");
    return BT_ERR_ARG;
  }
  BT_CUDA(cudaDeviceSynchronize());
  if (b->refined) return rbatch_status(b);
  int code = 0;
  BT_CUDA(cudaMemcpy(&code, reinterpret_cast<int*>(b->d_ctl) + 2, sizeof(int), cudaMemcpyDeviceToHost));
  if (code != 0) {
    set_error("bt_batch: a grid-barrier wait of the persistent launch gave up");
    return BT_ERR_TIMEOUT;
  }
  return BT_OK;
}

bt_status bt_batch_debug(bt_batch b, double limit_s, int32_t skip_stage) {
  if (!b || !(limit_s >= 0.0) || limit_s > 60.0 || skip_stage < -1) {
    set_error("bt_batch_debug: need a plan, 0 <= limit_s <= 60 and skip_stage >= -1");
    return BT_ERR_ARG;
  }
  if (b->refined) {
    set_error("bt_batch_debug: refined plans have no grid barrier");
    return BT_ERR_UNSUPPORTED;
  }
  return batch_set_debug(b, (unsigned long long)(limit_s * 1e9), skip_stage);
}

bt_status bt_batch_query(bt_batch b, int64_t out[6]) {
  if (!b || !out) {
    set_error("bt_batch_query: NULL argument");
    return BT_ERR_ARG;
  }
  if (b->refined) {
    out[0] = (int64_t)b->groups.size();
    out[1] = out[2] = out[3] = 0;
    out[4] = b->ropts.k_tile;
  } else {
    out[0] = b->n_items;
    out[1] = b->n_stages;
    out[2] = b->grid;
    out[3] = b->threads;
    out[4] = b->k_tile;
  }
  out[5] = b->exec ? 1 : 0;
  return BT_OK;
}

bt_status bt_batch_info(bt_batch b, int32_t i, bt_info* out) {
  if (!b || !out || i < 0 || i >= b->n) {
    set_error("bt_batch_info: need a plan, 0 <= i < n and an output");
    return BT_ERR_ARG;
  }
  if (!b->refined) {
    out->iters = 0;
    out->converged = 1;
    out->rel_res = -1.0;
    out->rel_res0 = -1.0;
    return BT_OK;
  }
  if (!b->infos_ready) {
    set_error("bt_batch_info: call bt_batch_status after the run first");
    return BT_ERR_ARG;
  }
  *out = b->infos[(size_t)b->set_group[(size_t)i]];
  return BT_OK;
}

void bt_batch_destroy(bt_batch b) { destroy_batch(b); }

bt_status bt_solve_batched(int32_t n, const bt_handle* h, const double* const* F, const int64_t* K,
                           double* const* X, const bt_opts* opts) {
  bt_batch b = nullptr;
  BT_TRY(bt_batch_create(n, h, F, K, X, opts, &b));
  bt_status st = bt_batch_run(b, opts ? opts->stream : nullptr);
  if (st == BT_OK) {
    cudaError_t e = cudaStreamSynchronize(opts ? (cudaStream_t)opts->stream : nullptr);
    if (e != cudaSuccess) st = cuda_fail(e, "bt_solve_batched");
  }
  if (st == BT_OK) st = bt_batch_status(b);
  destroy_batch(b);
  return st;
}


bt_status bt_handle_query(bt_handle h, int64_t out[6]) {
  if (!h || !out) {
    set_error("bt_handle_query: NULL argument");
    return BT_ERR_ARG;
  }
  out[0] = h->N;
  out[1] = h->M;
  out[2] = h->S;
  out[3] = h->depth;
  out[4] = h->stencil;
  out[5] = (int64_t)(h->arena.bytes + h->scratch_bytes);
  return BT_OK;
}

bt_status bt_handle_band(bt_handle h, int64_t out[5]) {
  if (!h || !out) {
    set_error("bt_handle_band: NULL argument");
    return BT_ERR_ARG;
  }
  for (int k = 0; k < 4; ++k) out[k] = h->band[k];
  out[4] = h->band_n;
  return BT_OK;
}

bt_status bt_factor_export(bt_handle h, int32_t what, double* dst) {
  if (!h || !dst || what < 0 || what > 5) {
    set_error("bt_factor_export: need a handle, a device buffer and what in 0..5");
    return BT_ERR_ARG;
  }
  if (what == 5) {
    cudaSetDevice(h->device);
    BT_TRY(factor_left_responses(h, nullptr));
  }
  const size_t MM = (size_t)h->M * h->M;
  const double* src = nullptr;
  size_t n = 0;
  switch (what) {
    case 0: src = h->U; n = h->N * MM; break;
    case 1: src = h->V; n = h->N * MM; break;
    case 2: src = h->At; n = h->S * MM; break;
    case 3: src = h->Ct; n = h->S * MM; break;
    case 4: src = h->Bt; n = h->S * MM; break;
    case 5: src = h->Y; n = h->N * MM; break;
  }
  BT_CUDA(cudaMemcpy(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice));
  return BT_OK;
}

bt_status bt_profile_enable(bt_handle h, int32_t enable) {
  if (!h) {
    set_error("bt_profile_enable: NULL handle");
    return BT_ERR_ARG;
  }
  h->prof.on = enable != 0;
  return BT_OK;
}

bt_status bt_profile_read(bt_handle h, bt_kernel_stat* out, int32_t cap, int32_t* n) {
  if (!h || !n || (cap > 0 && !out)) {
    set_error("bt_profile_read: NULL argument");
    return BT_ERR_ARG;
  }
  h->prof.collect();
  const int32_t cnt = (int32_t)h->prof.names.size();
  for (int32_t k = 0; k < cnt && k < cap; ++k) {
    std::memset(out[k].name, 0, sizeof(out[k].name));
    std::strncpy(out[k].name, h->prof.names[k].c_str(), sizeof(out[k].name) - 1);
    out[k].launches = h->prof.launches[k];
    out[k].total_ms = h->prof.total_ms[k];
  }
  *n = cnt;
  h->prof.names.clear();
  h->prof.launches.clear();
  h->prof.total_ms.clear();
  return BT_OK;
}

}  // extern "C"
