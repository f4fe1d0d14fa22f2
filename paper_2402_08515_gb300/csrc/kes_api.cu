// C ABI of the kes library: context, filter application and the Krylov
// eigensolver (Nannen & Wess, arXiv:2402.08515, Sec. 2).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <new>
#include <utility>
#include <vector>

#include "kes_internal.h"

using namespace kes;

namespace {

struct KesError {
  kes_status status;
};

#define KES_CUDA(call)                                              \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) {                                        \
      throw KesError{e_ == cudaErrorMemoryAllocation ? KES_ERR_OOM  \
                                                     : KES_ERR_CUDA}; \
    }                                                               \
  } while (0)

#define KES_CHECK_LAUNCH() KES_CUDA(cudaGetLastError())

template <typename F>
kes_status guarded(F&& f) {
  try {
    return f();
  } catch (const KesError& e) {
    return e.status;
  } catch (const std::bad_alloc&) {
    return KES_ERR_OOM;
  } catch (...) {
    return KES_ERR_CUDA;
  }
}

}  // namespace

struct kes_ctx {
  kes_opts opts{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int64_t n = 0, n_pad = 0, nnz = 0;
  double gershgorin = 0.0;    // sqrt(max_i sum_j |s_ij| / m_i) >= omega_max(S, M)
  double omega_est = 0.0;     // last power-iteration estimate (0: none)
  std::vector<std::pair<void*, size_t>> allocs;
  SellDev A;
  LaunchCfg cfg;
  int64_t nnz_pad = 0;
  int32_t* perm = nullptr;    // device; null = identity order
  double* m64 = nullptr;      // lumped mass (n_pad, zero padded)
  double* minv64 = nullptr;   // 1 / m (n_pad, zero padded)
  double* tau2m64 = nullptr;  // tau^2 / m (FP64 form)
  float* tau2m32 = nullptr;   // tau^2 / m (FP32 form)
  // filter
  bool filter_set = false;
  int F = 0, L = 0;
  double tau = 0.0;
  std::vector<double> wmin, wmax, h_alpha;
  double* alpha64 = nullptr;
  float* alpha_hi = nullptr;
  float* alpha_lo = nullptr;
  size_t alpha_cap = 0;
  // filter work
  double* stage_in = nullptr;   // n_pad, permuted start vector of the trajectory
  double* stage_out = nullptr;  // F x n_pad, filtered vectors (FP64)
  int stage_out_F = 0;
  double* U64[2] = {nullptr, nullptr};
  float* U32[3] = {nullptr, nullptr, nullptr};
  float* acc_s = nullptr;
  float* acc_c = nullptr;
  double* tmp = nullptr;        // n_pad scratch for host transfers / permutation
  int* d_flag = nullptr;
  // graph of one filter application
  cudaGraphExec_t gexec = nullptr;
  int g_F = -1, g_L = -1;
  int64_t g_nodes = 0;
  // Krylov workspace
  int kcap = 0;
  double* B = nullptr;
  double* SB = nullptr;
  double* Hd = nullptr;         // kcap x kcap col-major, column j holds b_i^T S b_j for i <= j
  double* partial = nullptr;
  double* scal = nullptr;       // device scalars
  double* Yd = nullptr;
  double* thd = nullptr;
  double* Xd = nullptr;
  size_t Xd_cap = 0;
  // stats
  kes_stats stats{};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_filter, ev_other;
  std::vector<cudaEvent_t> ev_pool;

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (opts.dev_alloc) {
      p = opts.dev_alloc(bytes, opts.alloc_user);
      if (!p) throw KesError{KES_ERR_OOM};
    } else {
      cudaError_t e = cudaMalloc(&p, bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        throw KesError{KES_ERR_OOM};
      }
    }
    allocs.emplace_back(p, bytes);
    return p;
  }
  void dfree(void* p) {
    if (!p) return;
    for (size_t i = 0; i < allocs.size(); ++i)
      if (allocs[i].first == p) {
        if (opts.dev_free) opts.dev_free(p, allocs[i].second, opts.alloc_user);
        else cudaFree(p);
        allocs.erase(allocs.begin() + i);
        return;
      }
  }
  template <typename T>
  T* dalloc_n(int64_t count) { return static_cast<T*>(dalloc(static_cast<size_t>(count) * sizeof(T))); }

  cudaEvent_t get_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    KES_CUDA(cudaEventCreate(&e));
    return e;
  }
  // Completes pending event pairs (the stream must have been synchronised).
  void harvest_events() {
    for (auto* list : {&ev_filter, &ev_other}) {
      for (auto& pr : *list) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
          if (list == &ev_filter) stats.filter_ms += ms;
          else stats.solve_other_ms += ms;
        }
        ev_pool.push_back(pr.first);
        ev_pool.push_back(pr.second);
      }
      list->clear();
    }
  }
  void sync() {
    KES_CUDA(cudaStreamSynchronize(stream));
    harvest_events();
  }
};

namespace {

void release(kes_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->harvest_events();
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  while (!c->allocs.empty()) c->dfree(c->allocs.back().first);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

// --------------------------------------------------------------- transfers
// Brings a length-n user vector (host or device, original order) into dst (n_pad, permuted order).
void vec_in(kes_ctx* c, const double* src, int32_t mem, double* dst) {
  double* target = c->perm ? c->tmp : dst;
  if (mem == KES_MEM_HOST)
    KES_CUDA(cudaMemcpyAsync(target, src, c->n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  else
    KES_CUDA(cudaMemcpyAsync(target, src, c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  if (c->perm) {
    launch_permute(c->stream, c->tmp, dst, c->perm, c->n, true);
    KES_CHECK_LAUNCH();
  }
}

// Copies src (n_pad, permuted order) out to a length-n user vector (host or device).
void vec_out(kes_ctx* c, const double* src, double* dst, int32_t mem) {
  const double* from = src;
  if (c->perm) {
    launch_permute(c->stream, src, c->tmp, c->perm, c->n, false);
    KES_CHECK_LAUNCH();
    from = c->tmp;
  }
  KES_CUDA(cudaMemcpyAsync(dst, from, c->n * sizeof(double),
                           mem == KES_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
}

// --------------------------------------------------------------- filter
// Issues the L fused steps of one filter application on c->stream:
// stage_in (one permuted vector) -> stage_out (F filtered vectors).
int64_t issue_filter_steps(kes_ctx* c) {
  const int64_t before = g_launches;
  const int L = c->L, F = c->F;
  if (c->opts.precision == KES_PREC_FP64) {
    for (int s = 0; s < L; ++s) {
      const bool first = s == 0, last = s == L - 1;
      const double* x = s == 0 ? c->stage_in : c->U64[(s - 1) & 1];
      const double* prev = s <= 1 ? c->stage_in : c->U64[s & 1];
      double* out = c->U64[s & 1];
      launch_step_f64(c->A, c->cfg, c->stream, first, c->tau2m64, x, prev, out, c->stage_out, c->n_pad, F,
                      c->alpha64, L, s, last, c->d_flag);
    }
  } else {
    launch_init_f32(c->stream, c->n_pad, c->stage_in, c->U32[2], c->acc_s, c->acc_c, c->n_pad, F, c->alpha64, L);
    for (int s = 0; s < L; ++s) {
      const bool first = s == 0, last = s == L - 1;
      const float* x = s == 0 ? c->U32[2] : c->U32[(s - 1) & 1];
      const float* prev = s <= 1 ? c->U32[2] : c->U32[s & 1];
      float* out = c->U32[s & 1];
      launch_step_f32(c->A, c->cfg, c->stream, first, last, c->tau2m32, x, prev, out, c->acc_s, c->acc_c,
                      c->stage_out, c->n_pad, F, c->alpha_hi, c->alpha_lo, L, s, c->d_flag);
    }
  }
  return g_launches - before;
}

void run_filter(kes_ctx* c) {
  cudaEvent_t e0 = c->get_event(), e1 = c->get_event();
  KES_CUDA(cudaEventRecord(e0, c->stream));
  if (c->opts.use_graph) {
    if (!c->gexec || c->g_F != c->F || c->g_L != c->L) {
      if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
      }
      cudaGraph_t graph;
      KES_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      const int64_t nodes = issue_filter_steps(c);
      cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
      g_launches -= nodes;  // captured, not launched
      KES_CUDA(ce);
      ce = cudaGraphInstantiate(&c->gexec, graph, 0);
      cudaGraphDestroy(graph);
      KES_CUDA(ce);
      c->g_F = c->F;
      c->g_L = c->L;
      c->g_nodes = nodes;
    }
    KES_CUDA(cudaGraphLaunch(c->gexec, c->stream));
    c->stats.kernel_launches += c->g_nodes;
  } else {
    c->stats.kernel_launches += issue_filter_steps(c);
    KES_CHECK_LAUNCH();
  }
  KES_CUDA(cudaEventRecord(e1, c->stream));
  c->ev_filter.emplace_back(e0, e1);
  c->stats.filter_calls += 1;
  c->stats.filter_steps += c->L;
}

void ensure_stage_out(kes_ctx* c, int F) {
  if (c->stage_out_F >= F) return;
  c->dfree(c->stage_out);
  c->stage_out = c->dalloc_n<double>(static_cast<int64_t>(F) * c->n_pad);
  KES_CUDA(cudaMemsetAsync(c->stage_out, 0, static_cast<size_t>(F) * c->n_pad * sizeof(double), c->stream));
  if (c->opts.precision == KES_PREC_FP32) {
    c->dfree(c->acc_s);
    c->dfree(c->acc_c);
    c->acc_s = c->dalloc_n<float>(static_cast<int64_t>(F) * c->n_pad);
    c->acc_c = c->dalloc_n<float>(static_cast<int64_t>(F) * c->n_pad);
    KES_CUDA(cudaMemsetAsync(c->acc_s, 0, static_cast<size_t>(F) * c->n_pad * sizeof(float), c->stream));
    KES_CUDA(cudaMemsetAsync(c->acc_c, 0, static_cast<size_t>(F) * c->n_pad * sizeof(float), c->stream));
  }
  c->stage_out_F = F;
  if (c->gexec) {  // buffers moved: recapture
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
}

kes_status check_flag(kes_ctx* c) {
  int flag = 0;
  KES_CUDA(cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  c->sync();
  if (flag) {
    KES_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
    return KES_ERR_UNSTABLE;
  }
  return KES_OK;
}

// --------------------------------------------------------------- Krylov workspace
void ensure_krylov(kes_ctx* c, int kmax) {
  if (c->kcap >= kmax) return;
  for (double* p : {c->B, c->SB, c->Hd, c->partial, c->scal, c->Yd, c->thd}) c->dfree(p);
  c->kcap = kmax;
  c->B = c->dalloc_n<double>(static_cast<int64_t>(kmax) * c->n_pad);
  c->SB = c->dalloc_n<double>(static_cast<int64_t>(kmax) * c->n_pad);
  c->Hd = c->dalloc_n<double>(static_cast<int64_t>(kmax) * kmax);
  c->partial = c->dalloc_n<double>(static_cast<int64_t>(kDotBlocks) * (2 * kmax + 8));
  c->scal = c->dalloc_n<double>(2 * kmax + 16);
  c->Yd = c->dalloc_n<double>(static_cast<int64_t>(kmax) * kmax);
  c->thd = c->dalloc_n<double>(kmax);
  KES_CUDA(cudaMemsetAsync(c->Hd, 0, sizeof(double) * kmax * kmax, c->stream));
}

// Times every launch shape of the step kernel on this matrix (a few steps on zeroed
// scratch state, CUDA events) and keeps the fastest. All shapes compute the same sums.
void tune_step(kes_ctx* c) {
  const bool fp32 = c->opts.precision == KES_PREC_FP32;
  const int nv = step_variant_count();
  ensure_stage_out(c, 1);
  double* a64 = c->dalloc_n<double>(8);
  float* a32 = c->dalloc_n<float>(8);
  KES_CUDA(cudaMemsetAsync(a64, 0, 8 * sizeof(double), c->stream));
  KES_CUDA(cudaMemsetAsync(a32, 0, 8 * sizeof(float), c->stream));
  cudaEvent_t e0 = c->get_event(), e1 = c->get_event();
  auto steps = [&](int count) {
    for (int i = 0; i < count; ++i) {
      if (fp32)
        launch_step_f32(c->A, c->cfg, c->stream, false, false, c->tau2m32, c->U32[0], c->U32[1], c->U32[1],
                        c->acc_s, c->acc_c, c->stage_out, c->n_pad, 1, a32, a32, 7, 1, c->d_flag);
      else
        launch_step_f64(c->A, c->cfg, c->stream, false, c->tau2m64, c->U64[0], c->U64[1], c->U64[1],
                        c->stage_out, c->n_pad, 1, a64, 7, 1, false, c->d_flag);
    }
  };
  int best = 0;
  float best_ms = 3.0e38f;
  for (int v = 0; v < nv; ++v) {
    c->cfg.variant = v;
    c->cfg.grid_step = c->cfg.n_sm * step_blocks_per_sm(fp32, v, c->cfg.block_step);
    steps(2);
    float ms_v = 3.0e38f;
    for (int rep = 0; rep < 2; ++rep) {
      KES_CUDA(cudaEventRecord(e0, c->stream));
      steps(6);
      KES_CUDA(cudaEventRecord(e1, c->stream));
      KES_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      KES_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      ms_v = std::min(ms_v, ms);
    }
    KES_CHECK_LAUNCH();
    if (ms_v < best_ms) {
      best_ms = ms_v;
      best = v;
    }
  }
  c->ev_pool.push_back(e0);
  c->ev_pool.push_back(e1);
  c->cfg.variant = best;
  c->cfg.grid_step = c->cfg.n_sm * step_blocks_per_sm(fp32, best, c->cfg.block_step);
  c->sync();
  c->dfree(a64);
  c->dfree(a32);
}

void validate_csr(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val, const double* m) {
  if (n <= 0 || n >= (int64_t(1) << 31) || !row_ptr || !col || !val || !m) throw KesError{KES_ERR_ARG};
  if (row_ptr[0] != 0) throw KesError{KES_ERR_ARG};
  for (int64_t i = 0; i < n; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) throw KesError{KES_ERR_ARG};
    int64_t last = -1;
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      if (col[p] < 0 || col[p] >= n || col[p] <= last) throw KesError{KES_ERR_ARG};
      if (!std::isfinite(val[p])) throw KesError{KES_ERR_ARG};
      last = col[p];
    }
    if (!(m[i] > 0.0) || !std::isfinite(m[i])) throw KesError{KES_ERR_MASS};
  }
}

}  // namespace

// =========================================================================
// C ABI
// =========================================================================
extern "C" {

void kes_opts_default(kes_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = KES_PREC_FP64;
  o->sell_sigma = 1;
  o->use_graph = 1;
  o->block_b = 1;
  o->autotune = 1;
}

void kes_solve_opts_default(kes_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->kmax = 40;
  o->check_every = 5;
  o->n_wanted = 0;
  o->want_vectors = 0;
  o->tol = 1e-8;
}

const char* kes_strerror(int32_t s) {
  switch (s) {
    case KES_OK: return "ok";
    case KES_INFO_INVARIANT_SUBSPACE: return "Krylov breakdown: invariant subspace found";
    case KES_ERR_ARG: return "invalid argument";
    case KES_ERR_MASS: return "lumped mass entry not positive or not finite";
    case KES_ERR_UNSTABLE: return "time stepping unstable (CFL violated or non-finite state)";
    case KES_ERR_CUDA: return "CUDA runtime error";
    case KES_ERR_OOM: return "out of memory";
    case KES_ERR_TIMEOUT: return "device wait timed out";
    case KES_ERR_STATE: return "call out of order";
    case KES_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

kes_status kes_create(kes_ctx** out, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                      const double* m_diag, const kes_opts* opts) {
  if (!out) return KES_ERR_ARG;
  *out = nullptr;
  kes_ctx* c = nullptr;
  kes_status st = guarded([&]() -> kes_status {
    validate_csr(n, row_ptr, col, val, m_diag);
    c = new kes_ctx();
    if (opts) c->opts = *opts;
    else kes_opts_default(&c->opts);
    if (c->opts.precision != KES_PREC_FP64 && c->opts.precision != KES_PREC_FP32) throw KesError{KES_ERR_ARG};
    if (c->opts.sell_sigma < 1) c->opts.sell_sigma = 1;
    if (c->opts.block_b < 1) c->opts.block_b = 1;
    if ((c->opts.dev_alloc == nullptr) != (c->opts.dev_free == nullptr)) throw KesError{KES_ERR_ARG};
    KES_CUDA(cudaGetDevice(&c->device));
    int n_sm = 0;
    KES_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device));
    if (c->opts.stream) {
      c->stream = static_cast<cudaStream_t>(c->opts.stream);
    } else {
      KES_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    c->n = n;
    c->nnz = row_ptr[n];
    // Gershgorin bound of M^{-1} S
    double g = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) s += std::fabs(val[p]);
      g = std::max(g, s / m_diag[i]);
    }
    c->gershgorin = std::sqrt(g);

    SellHost sh = build_sell(n, row_ptr, col, val, c->opts.sell_sigma);
    c->n_pad = sh.n_slices * kSliceC;
    c->nnz_pad = sh.nnz_pad;
    int64_t* sp = c->dalloc_n<int64_t>(sh.n_slices + 1);
    int32_t* dc = c->dalloc_n<int32_t>(sh.nnz_pad);
    KES_CUDA(cudaMemcpyAsync(sp, sh.slice_ptr.data(), (sh.n_slices + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                             c->stream));
    KES_CUDA(cudaMemcpyAsync(dc, sh.col.data(), sh.nnz_pad * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    c->A.n = n;
    c->A.n_pad = c->n_pad;
    c->A.n_slices = sh.n_slices;
    c->A.slice_ptr = sp;
    c->A.col = dc;
    // FP64 values are always kept: the Krylov basis needs S b_k in FP64
    double* dv = c->dalloc_n<double>(sh.nnz_pad);
    KES_CUDA(cudaMemcpyAsync(dv, sh.val.data(), sh.nnz_pad * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->A.val64 = dv;
    if (c->opts.precision == KES_PREC_FP32) {
      std::vector<float> v32(sh.val.begin(), sh.val.end());
      float* dv32 = c->dalloc_n<float>(sh.nnz_pad);
      KES_CUDA(cudaMemcpyAsync(dv32, v32.data(), sh.nnz_pad * sizeof(float), cudaMemcpyHostToDevice, c->stream));
      c->A.val32 = dv32;
      c->sync();  // v32 goes out of scope
    }
    if (!sh.perm.empty()) {
      c->perm = c->dalloc_n<int32_t>(n);
      KES_CUDA(cudaMemcpyAsync(c->perm, sh.perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    }
    // per-row vectors in permuted order, zero padded
    std::vector<double> mp(c->n_pad, 0.0), minv(c->n_pad, 0.0);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t o = sh.perm.empty() ? i : sh.perm[i];
      mp[i] = m_diag[o];
      minv[i] = 1.0 / m_diag[o];
    }
    c->m64 = c->dalloc_n<double>(c->n_pad);
    c->minv64 = c->dalloc_n<double>(c->n_pad);
    KES_CUDA(cudaMemcpyAsync(c->m64, mp.data(), c->n_pad * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    KES_CUDA(cudaMemcpyAsync(c->minv64, minv.data(), c->n_pad * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->tau2m64 = c->dalloc_n<double>(c->n_pad);
    KES_CUDA(cudaMemsetAsync(c->tau2m64, 0, c->n_pad * sizeof(double), c->stream));
    if (c->opts.precision == KES_PREC_FP32) {
      c->tau2m32 = c->dalloc_n<float>(c->n_pad);
      for (int j = 0; j < 3; ++j) {
        c->U32[j] = c->dalloc_n<float>(c->n_pad);
        KES_CUDA(cudaMemsetAsync(c->U32[j], 0, c->n_pad * sizeof(float), c->stream));
      }
    } else {
      for (int j = 0; j < 2; ++j) {
        c->U64[j] = c->dalloc_n<double>(c->n_pad);
        KES_CUDA(cudaMemsetAsync(c->U64[j], 0, c->n_pad * sizeof(double), c->stream));
      }
    }
    c->stage_in = c->dalloc_n<double>(c->n_pad);
    c->tmp = c->dalloc_n<double>(c->n_pad);
    KES_CUDA(cudaMemsetAsync(c->stage_in, 0, c->n_pad * sizeof(double), c->stream));
    c->d_flag = c->dalloc_n<int>(4);
    KES_CUDA(cudaMemsetAsync(c->d_flag, 0, 4 * sizeof(int), c->stream));
    if (c->tau2m32) KES_CUDA(cudaMemsetAsync(c->tau2m32, 0, c->n_pad * sizeof(float), c->stream));
    // grid-stride launch shape: one full wave of resident 256-thread blocks
    c->cfg.n_sm = n_sm;
    c->cfg.block_step = 256;
    if (c->opts.step_variant < 0 || c->opts.step_variant >= step_variant_count()) throw KesError{KES_ERR_ARG};
    c->cfg.variant = c->opts.step_variant;
    c->cfg.grid_step =
        n_sm * step_blocks_per_sm(c->opts.precision == KES_PREC_FP32, c->cfg.variant, c->cfg.block_step);
    if (c->opts.autotune) tune_step(c);
    c->sync();
    c->stats.bytes_per_step = kes_step_bytes(c, 1, 1);
    c->stats.step_variant = c->cfg.variant;
    c->stats.step_grid = c->cfg.grid_step;
    return KES_OK;
  });
  if (st != KES_OK) {
    release(c);
    return st;
  }
  *out = c;
  return KES_OK;
}

void kes_destroy(kes_ctx* ctx) { release(ctx); }

int64_t kes_size(const kes_ctx* ctx) { return ctx ? ctx->n : -1; }

kes_status kes_sync(kes_ctx* ctx) {
  if (!ctx) return KES_ERR_ARG;
  return guarded([&]() -> kes_status { return check_flag(ctx); });
}

int64_t kes_step_bytes(const kes_ctx* c, int32_t b, int32_t F) {
  if (!c || b < 1 || F < 1) return -1;
  // matrix: value + int32 column per stored entry; per row and vector: gather of u_n once,
  // tau^2/m, u_{n-1} read, u_{n+1} written, F accumulators read and written.
  if (c->opts.precision == KES_PREC_FP64)
    return 12 * c->nnz + 4 * (c->n + 1) + c->n * (8 + int64_t(b) * (8 + 8 + 8 + 16 * F));
  return 8 * c->nnz + c->n * (4 + int64_t(b) * (4 + 4 + 4 + 16 * F));
}

kes_status kes_estimate_omega_max(kes_ctx* c, int32_t iters, const double* v0, double* omega_max,
                                  double* gershgorin) {
  if (!c || !v0 || !omega_max || iters < 0) return KES_ERR_ARG;
  return guarded([&]() -> kes_status {
    const int64_t launches0 = g_launches;
    ensure_krylov(c, 2);
    double* v = c->U64[0] ? c->U64[0] : c->B;  // scratch n_pad vectors
    double* w = c->U64[1] ? c->U64[1] : c->SB;
    KES_CUDA(cudaMemsetAsync(v, 0, c->n_pad * sizeof(double), c->stream));
    KES_CUDA(cudaMemsetAsync(w, 0, c->n_pad * sizeof(double), c->stream));
    vec_in(c, v0, KES_MEM_HOST, w);
    launch_mdot(c->stream, w, 0, 1, w, nullptr, c->n_pad, c->partial, c->scal);
    launch_scale_rsqrt(c->stream, w, c->scal, v, nullptr, c->n_pad);
    for (int it = 0; it < iters; ++it) {
      launch_spmv_f64(c->A, c->cfg, c->stream, v, c->minv64, w);
      launch_mdot(c->stream, w, 0, 1, w, nullptr, c->n_pad, c->partial, c->scal);
      launch_scale_rsqrt(c->stream, w, c->scal, v, nullptr, c->n_pad);
    }
    launch_spmv_f64(c->A, c->cfg, c->stream, v, nullptr, w);
    launch_mdot(c->stream, v, 0, 1, w, nullptr, c->n_pad, c->partial, c->scal);          // v^T S v
    launch_mdot(c->stream, v, 0, 1, v, c->m64, c->n_pad, c->partial, c->scal + 1);      // v^T M v
    KES_CHECK_LAUNCH();
    double h[2];
    KES_CUDA(cudaMemcpyAsync(h, c->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    c->sync();
    c->stats.kernel_launches += g_launches - launches0;
    *omega_max = std::sqrt(std::max(h[0], 0.0) / h[1]);
    c->omega_est = *omega_max;
    if (gershgorin) *gershgorin = c->gershgorin;
    return KES_OK;
  });
}

kes_status kes_set_filters(kes_ctx* c, int32_t F, const double* wmin, const double* wmax, double tau, int32_t L) {
  if (!c || F < 1 || !wmin || !wmax || !(tau > 0.0) || L < 1 || !std::isfinite(tau)) return KES_ERR_ARG;
  for (int f = 0; f < F; ++f)
    if (!(wmin[f] >= 0.0) || !(wmax[f] > wmin[f]) || !std::isfinite(wmax[f])) return KES_ERR_ARG;
  if (c->omega_est > 0.0 && tau * c->omega_est >= 2.0) return KES_ERR_UNSTABLE;
  return guarded([&]() -> kes_status {
    const size_t need = static_cast<size_t>(F) * (L + 1);
    c->h_alpha.assign(need, 0.0);
    for (int f = 0; f < F; ++f) alpha_table(wmin[f], wmax[f], tau, L, c->h_alpha.data() + f * (L + 1));
    c->sync();
    if (need > c->alpha_cap) {
      c->dfree(c->alpha64);
      c->dfree(c->alpha_hi);
      c->dfree(c->alpha_lo);
      c->alpha64 = c->dalloc_n<double>(need);
      c->alpha_hi = c->dalloc_n<float>(need);
      c->alpha_lo = c->dalloc_n<float>(need);
      c->alpha_cap = need;
      if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
      }
    }
    std::vector<float> hi(need), lo(need);
    for (size_t i = 0; i < need; ++i) {
      hi[i] = static_cast<float>(c->h_alpha[i]);
      lo[i] = static_cast<float>(c->h_alpha[i] - static_cast<double>(hi[i]));
    }
    KES_CUDA(cudaMemcpyAsync(c->alpha64, c->h_alpha.data(), need * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    KES_CUDA(cudaMemcpyAsync(c->alpha_hi, hi.data(), need * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    KES_CUDA(cudaMemcpyAsync(c->alpha_lo, lo.data(), need * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    // tau^2 / m in permuted order
    std::vector<double> m(c->n_pad);
    KES_CUDA(cudaMemcpyAsync(m.data(), c->m64, c->n_pad * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    c->sync();
    std::vector<double> t2m(c->n_pad, 0.0);
    for (int64_t i = 0; i < c->n; ++i) t2m[i] = tau * tau / m[i];
    KES_CUDA(cudaMemcpyAsync(c->tau2m64, t2m.data(), c->n_pad * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (c->tau2m32) {
      std::vector<float> t32(t2m.begin(), t2m.end());
      KES_CUDA(cudaMemcpyAsync(c->tau2m32, t32.data(), c->n_pad * sizeof(float), cudaMemcpyHostToDevice, c->stream));
      c->sync();
    }
    ensure_stage_out(c, F);
    c->sync();
    c->F = F;
    c->L = L;
    c->tau = tau;
    c->wmin.assign(wmin, wmin + F);
    c->wmax.assign(wmax, wmax + F);
    c->filter_set = true;
    return KES_OK;
  });
}

kes_status kes_set_filter(kes_ctx* c, double wmin, double wmax, double tau, int32_t L) {
  return kes_set_filters(c, 1, &wmin, &wmax, tau, L);
}

kes_status kes_alpha_table(double wmin, double wmax, double tau, int32_t L, double* alpha) {
  if (!alpha || L < 1 || !(tau > 0.0) || !(wmax > wmin) || !(wmin >= 0.0)) return KES_ERR_ARG;
  kes::alpha_table(wmin, wmax, tau, L, alpha);
  return KES_OK;
}

kes_status kes_filter_response(double wmin, double wmax, double tau, int32_t L, const double* omega, int64_t k,
                               double* beta) {
  if (!omega || !beta || k < 0 || L < 1 || !(tau > 0.0) || !(wmax > wmin) || !(wmin >= 0.0)) return KES_ERR_ARG;
  kes::filter_response(wmin, wmax, tau, L, omega, k, beta);
  return KES_OK;
}

kes_status kes_sym_eig(int32_t k, const double* A, double* w, double* V) {
  if (k < 0 || (k > 0 && (!A || !w))) return KES_ERR_ARG;
  return kes::sym_eig(k, A, w, V) ? KES_OK : KES_ERR_ARG;
}

kes_status kes_filter_apply(kes_ctx* c, const double* r_in, double* r_out, int32_t b, int32_t mem) {
  if (!c || !r_in || !r_out || b < 1 || b > c->opts.block_b || (mem != KES_MEM_HOST && mem != KES_MEM_DEVICE))
    return KES_ERR_ARG;
  if (!c->filter_set) return KES_ERR_STATE;
  return guarded([&]() -> kes_status {
    for (int j = 0; j < b; ++j) {
      vec_in(c, r_in + static_cast<int64_t>(j) * c->n, mem, c->stage_in);
      run_filter(c);
      for (int f = 0; f < c->F; ++f)
        vec_out(c, c->stage_out + static_cast<int64_t>(f) * c->n_pad,
                r_out + (static_cast<int64_t>(f) * b + j) * c->n, mem);
    }
    KES_CHECK_LAUNCH();
    if (mem == KES_MEM_HOST) return check_flag(c);
    return KES_OK;
  });
}

void kes_result_free(kes_result* r) {
  if (!r) return;
  std::free(r->omega2);
  std::free(r->omega);
  std::free(r->rel_res);
  std::free(r->abs_res);
  std::free(r->vectors);
  std::free(r->ritz_omega2);
  std::free(r->ritz_rel_res);
  std::free(r);
}

kes_status kes_krylov_solve(kes_ctx* c, const double* r0, int32_t mem, const kes_solve_opts* so_in,
                            kes_result** out) {
  if (!c || !r0 || !out || (mem != KES_MEM_HOST && mem != KES_MEM_DEVICE)) return KES_ERR_ARG;
  *out = nullptr;
  if (!c->filter_set) return KES_ERR_STATE;
  if (c->F != 1) return KES_ERR_UNSUPPORTED;
  kes_solve_opts so;
  if (so_in) so = *so_in;
  else kes_solve_opts_default(&so);
  if (so.kmax < 1 || so.check_every < 1 || !(so.tol > 0.0)) return KES_ERR_ARG;
  const auto t_start = std::chrono::steady_clock::now();
  kes_result* res = static_cast<kes_result*>(std::calloc(1, sizeof(kes_result)));
  if (!res) return KES_ERR_OOM;
  kes_status st = guarded([&]() -> kes_status {
    const int kmax = so.kmax;
    ensure_krylov(c, kmax);
    const int64_t np = c->n_pad;
    const double wmin = c->wmin[0], wmax = c->wmax[0];
    cudaStream_t s = c->stream;
    double* B = c->B;
    double* SB = c->SB;
    double* w = c->stage_out;  // the filtered vector is orthogonalised in place
    auto other_begin = [&]() {
      cudaEvent_t e0 = c->get_event();
      KES_CUDA(cudaEventRecord(e0, s));
      return e0;
    };
    auto other_end = [&](cudaEvent_t e0) {
      cudaEvent_t e1 = c->get_event();
      KES_CUDA(cudaEventRecord(e1, s));
      c->ev_other.emplace_back(e0, e1);
    };
    const int64_t launches0 = g_launches;

    // b_0 = r0 / ||r0||_M ; S b_0 ; H(0,0)
    cudaEvent_t e0 = other_begin();
    vec_in(c, r0, mem, c->stage_in);
    launch_mdot(s, c->stage_in, 0, 1, c->stage_in, c->m64, np, c->partial, c->scal);
    launch_scale_rsqrt(s, c->stage_in, c->scal, B, c->stage_in, np);
    launch_spmv_f64(c->A, c->cfg, s, B, nullptr, SB);
    launch_mdot(s, B, np, 1, SB, nullptr, np, c->partial, c->Hd);
    KES_CHECK_LAUNCH();
    other_end(e0);

    std::vector<double> Hh, theta, Y, rr;
    int k = 1;
    bool breakdown = false;
    int64_t steps = 0;
    // projection state of the last solve of eq. (projevp)
    std::vector<double> last_theta, last_rel;
    std::vector<int> acc_idx;
    std::vector<double> acc_theta, acc_rel, acc_abs, acc_Y;

    auto project = [&](int kk) {
      Hh.assign(static_cast<size_t>(kk) * kk, 0.0);
      KES_CUDA(cudaMemcpy2DAsync(Hh.data(), kk * sizeof(double), c->Hd, c->kcap * sizeof(double),
                                 kk * sizeof(double), kk, cudaMemcpyDeviceToHost, s));
      c->sync();
      // column j holds rows 0..j (upper triangle); mirror it into the lower triangle
      for (int j = 0; j < kk; ++j)
        for (int i = j + 1; i < kk; ++i) Hh[static_cast<size_t>(j) * kk + i] = Hh[static_cast<size_t>(i) * kk + j];
      theta.assign(kk, 0.0);
      Y.assign(static_cast<size_t>(kk) * kk, 0.0);
      if (!sym_eig(kk, Hh.data(), theta.data(), Y.data())) throw KesError{KES_ERR_CUDA};
      for (double& t : theta) t = std::max(t, 0.0);
      std::vector<int> inside;
      for (int j = 0; j < kk; ++j) {
        const double om = std::sqrt(theta[j]);
        if (om >= wmin && om <= wmax) inside.push_back(j);
      }
      const int p = static_cast<int>(inside.size());
      last_theta = theta;
      last_rel.assign(kk, std::numeric_limits<double>::quiet_NaN());
      acc_idx.clear();
      acc_theta.clear();
      acc_rel.clear();
      acc_abs.clear();
      acc_Y.clear();
      if (p == 0) return;
      std::vector<double> Ysel(static_cast<size_t>(kk) * p), thsel(p);
      for (int q = 0; q < p; ++q) {
        thsel[q] = theta[inside[q]];
        std::memcpy(&Ysel[static_cast<size_t>(q) * kk], &Y[static_cast<size_t>(inside[q]) * kk], kk * sizeof(double));
      }
      if (p > c->kcap) throw KesError{KES_ERR_ARG};
      cudaEvent_t ev = other_begin();
      KES_CUDA(cudaMemcpyAsync(c->Yd, Ysel.data(), Ysel.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      KES_CUDA(cudaMemcpyAsync(c->thd, thsel.data(), p * sizeof(double), cudaMemcpyHostToDevice, s));
      launch_ritz_residual(s, B, SB, np, kk, c->Yd, c->thd, p, c->m64, np, c->partial, c->scal);
      KES_CHECK_LAUNCH();
      rr.assign(2 * p, 0.0);
      KES_CUDA(cudaMemcpyAsync(rr.data(), c->scal, 2 * p * sizeof(double), cudaMemcpyDeviceToHost, s));
      other_end(ev);
      c->sync();
      for (int q = 0; q < p; ++q) {
        const double a = std::sqrt(std::max(rr[q], 0.0));
        const double den = thsel[q] * std::sqrt(std::max(rr[p + q], 0.0));
        const double rel = den > 0.0 ? a / den : std::numeric_limits<double>::infinity();
        last_rel[inside[q]] = rel;
        if (rel <= so.tol) {
          acc_idx.push_back(inside[q]);
          acc_theta.push_back(thsel[q]);
          acc_rel.push_back(rel);
          acc_abs.push_back(a);
          acc_Y.insert(acc_Y.end(), Ysel.begin() + static_cast<size_t>(q) * kk,
                       Ysel.begin() + static_cast<size_t>(q + 1) * kk);
        }
      }
    };

    int kproj = 0;
    while (k < kmax) {
      run_filter(c);  // stage_in = b_{k-1} -> w = C b_{k-1}
      steps += c->L;
      cudaEvent_t ev = other_begin();
      double* sc = c->scal;
      launch_mdot(s, w, 0, 1, w, c->m64, np, c->partial, sc);          // ||w||_M^2 before
      for (int pass = 0; pass < 2; ++pass) {
        launch_mdot(s, B, np, k, w, c->m64, np, c->partial, sc + 4);   // h = B^T M w
        launch_gemv_sub(s, w, B, np, k, sc + 4, np);                   // w -= B h
      }
      launch_mdot(s, w, 0, 1, w, c->m64, np, c->partial, sc + 1);      // ||w||_M^2 after
      KES_CHECK_LAUNCH();
      double nrm[2];
      int flag = 0;
      KES_CUDA(cudaMemcpyAsync(nrm, sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      KES_CUDA(cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      other_end(ev);
      c->sync();
      if (flag) {
        KES_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
        throw KesError{KES_ERR_UNSTABLE};
      }
      if (!(std::sqrt(nrm[1]) > 1e-10 * std::sqrt(nrm[0]))) {
        breakdown = true;
        break;
      }
      ev = other_begin();
      double* bk = B + static_cast<int64_t>(k) * np;
      double* sbk = SB + static_cast<int64_t>(k) * np;
      launch_scale_rsqrt(s, w, sc + 1, bk, c->stage_in, np);            // b_k, next filter input
      launch_spmv_f64(c->A, c->cfg, s, bk, nullptr, sbk);               // S b_k
      launch_mdot(s, B, np, k + 1, sbk, nullptr, np, c->partial, c->Hd + static_cast<int64_t>(k) * c->kcap);
      KES_CHECK_LAUNCH();
      other_end(ev);
      ++k;
      if (k % so.check_every == 0 && k < kmax) {
        project(k);
        kproj = k;
        if (so.n_wanted > 0 && static_cast<int>(acc_idx.size()) >= so.n_wanted) break;
      }
    }
    if (kproj != k) project(k);

    const int p = static_cast<int>(acc_idx.size());
    res->n = c->n;
    res->n_pairs = p;
    res->k_used = k;
    res->breakdown = breakdown ? 1 : 0;
    res->n_ritz = k;
    res->time_steps = steps;
    auto hdup = [](const std::vector<double>& v) {
      double* d = static_cast<double*>(std::malloc(std::max<size_t>(1, v.size()) * sizeof(double)));
      if (!d) throw std::bad_alloc();
      if (!v.empty()) std::memcpy(d, v.data(), v.size() * sizeof(double));
      return d;
    };
    res->omega2 = hdup(acc_theta);
    std::vector<double> om(p);
    for (int q = 0; q < p; ++q) om[q] = std::sqrt(acc_theta[q]);
    res->omega = hdup(om);
    res->rel_res = hdup(acc_rel);
    res->abs_res = hdup(acc_abs);
    res->ritz_omega2 = hdup(last_theta);
    res->ritz_rel_res = hdup(last_rel);
    if (so.want_vectors && p > 0) {
      const size_t need = static_cast<size_t>(p) * np;
      if (need > c->Xd_cap) {
        c->dfree(c->Xd);
        c->Xd = c->dalloc_n<double>(need);
        c->Xd_cap = need;
      }
      KES_CUDA(cudaMemcpyAsync(c->Yd, acc_Y.data(), acc_Y.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      launch_gemm_bx(s, B, np, k, c->Yd, p, c->Xd, np, np);
      KES_CHECK_LAUNCH();
      res->vectors = static_cast<double*>(std::malloc(static_cast<size_t>(p) * c->n * sizeof(double)));
      if (!res->vectors) throw std::bad_alloc();
      for (int q = 0; q < p; ++q) vec_out(c, c->Xd + static_cast<int64_t>(q) * np, res->vectors + q * c->n, KES_MEM_HOST);
    }
    c->sync();
    c->stats.kernel_launches += g_launches - launches0;
    return breakdown ? KES_INFO_INVARIANT_SUBSPACE : KES_OK;
  });
  res->solve_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (st != KES_OK && st != KES_INFO_INVARIANT_SUBSPACE) {
    kes_result_free(res);
    return st;
  }
  *out = res;
  return st;
}

kes_status kes_get_stats(kes_ctx* c, kes_stats* s) {
  if (!c || !s) return KES_ERR_ARG;
  return guarded([&]() -> kes_status {
    c->sync();
    *s = c->stats;
    return KES_OK;
  });
}

kes_status kes_reset_stats(kes_ctx* c) {
  if (!c) return KES_ERR_ARG;
  return guarded([&]() -> kes_status {
    c->sync();
    const int64_t bps = c->stats.bytes_per_step;
    c->stats = kes_stats{};
    c->stats.bytes_per_step = bps;
    c->stats.step_variant = c->cfg.variant;
    c->stats.step_grid = c->cfg.grid_step;
    return KES_OK;
  });
}

}  // extern "C"
