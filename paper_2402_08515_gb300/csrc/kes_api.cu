// C ABI of the kes library: context, filter application and the Krylov
// eigensolver (Nannen & Wess, arXiv:2402.08515, Sec. 2 and the block version of
// Sec. 4).
//
// A context holds one or several meshes (independent pencils) stacked
// block-diagonally: every mesh occupies a 32-row-aligned range of padded rows
// and of SELL slices, so that one launch per time step advances all of them.
// Each mesh keeps its own time step, weight tables, Krylov basis and
// projected problem.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include "kes_internal.h"

using namespace kes;

namespace {

struct KesError {
  kes_status status;
};

#define KES_CUDA(call)                                                \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) {                                          \
      throw KesError{e_ == cudaErrorMemoryAllocation ? KES_ERR_OOM    \
                                                     : KES_ERR_CUDA}; \
    }                                                                 \
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

struct MeshInfo {
  int64_t n = 0;          // dofs of this mesh
  int64_t n_pad = 0;      // its padded rows (multiple of 32)
  int64_t row_off = 0;    // first padded row in the context
  int64_t src_off = 0;    // first row in the caller's concatenated vectors
  int64_t slice_off = 0;  // first SELL slice
  int64_t n_slices = 0;
  int64_t nnz = 0;
  double gershgorin = 0;  // sqrt(max_i sum_j |s_ij| / m_i) >= omega_max
  double omega_est = 0;   // last power-iteration estimate (0: none)
  double tau = 0;
  std::vector<double> wmin, wmax;
};

// Adds the kernels launched while it lives (this thread) to the context's counter.
struct LaunchCount {
  kes_stats* stats;
  int64_t start;
  explicit LaunchCount(kes_stats* s) : stats(s), start(g_launches) {}
  ~LaunchCount() { stats->kernel_launches += g_launches - start; }
};

struct GraphEntry {
  int NB = 0;
  bool fp64 = true;
  int cpt = 0;
  int steps = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t nodes = 0;
};

int nb_for(int b) { return b <= 1 ? 1 : b <= 2 ? 2 : b <= 4 ? 4 : 8; }

}  // namespace

struct kes_ctx {
  kes_opts opts{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  std::vector<MeshInfo> meshes;
  int64_t n = 0, n_pad = 0, nnz = 0, nnz_pad = 0;
  std::vector<std::pair<void*, size_t>> allocs;
  SellDev A;
  LaunchCfg cfg;
  int NBcap = 1;
  int32_t* row_src = nullptr;     // padded row -> caller row (-1: padding); null: identity
  int32_t* slice_mesh = nullptr;  // slice -> mesh (null: one mesh)
  double* m64 = nullptr;          // lumped mass (n_pad, zero padded)
  double* minv64 = nullptr;       // 1 / m
  double* tau2m64 = nullptr;      // tau^2 / m with the tau of the row's mesh
  double* step64 = nullptr;       // A = -tau^2 M^{-1} S, SELL layout (FP64 steps)
  double* step64p = nullptr;      // the same in the pair layout (A.slice_ptr2); FP64 contexts with fold64
  float* step32 = nullptr;        // the same in FP32 (FP32 steps)
  float* step32p = nullptr;       // the FP32 ones in the pair layout (A.slice_ptr2), if built
  int64_t nnz_pair = 0;           // entries of the pair layout (with its padding)
  bool diag_in_rows = false;      // every row of the SELL layout stores its diagonal among its slice's
                                  // width (a real entry or padding): the 2 u_n can fold into A
  bool fold64 = false;            // the FP64 step values hold A + 2I (leapfrog and diag_in_rows)
  SellDev step_A64() const {
    SellDev a = A;
    a.val64 = step64;
    a.val64p = step64p;
    a.fold2 = fold64 ? 1 : 0;
    return a;
  }
  SellDev step_A32() const {
    SellDev a = A;
    a.val32 = step32;
    a.val32p = step32p;
    return a;
  }
  // filter
  bool filter_set = false;
  int F = 0, L = 0;
  double* alpha64 = nullptr;  // [n_mesh][F][L+1]
  float* alpha_hi = nullptr;
  float* alpha_lo = nullptr;
  size_t alpha_cap = 0;
  // filter work (capacity NBcap columns)
  double* stage_in = nullptr;   // n_pad x NB row-major: the start block of the trajectory
  double* stage_out = nullptr;  // F x (n_pad x NB): filtered blocks (FP64)
  int stage_out_F = 0;
  double* U64[2] = {nullptr, nullptr};
  float* U32[3] = {nullptr, nullptr, nullptr};
  double* V64 = nullptr;  // fourth-order stage v = u + A u / 12 (n_pad x NBcap), allocated on first use
  float* V32 = nullptr;
  float* acc_s = nullptr;
  float* acc_c = nullptr;
  double* tmp_user = nullptr;  // n x NBcap, caller layout
  int* d_flag = nullptr;
  std::vector<GraphEntry> graphs;
  int g_F = -1, g_L = -1;
  // Krylov workspace
  int kcap = 0, kF = 0;  // basis vectors per process, intervals (processes per mesh)
  double* B = nullptr;   // n_pad x (kF * kcap), column-major: interval f owns columns f * kcap ..,
                         // mesh j its rows row_off_j ..
  double* SB = nullptr;
  double* Hd = nullptr;  // (n_mesh * kF) x kcap x kcap; column k of process p holds b_i^T S b_k, i <= k
  double* partial = nullptr;
  double* scal = nullptr;  // per process: 2 * kcap + kScal device scalars
  double* normd = nullptr; // per process: ||w||_M^2 before and after orthogonalisation
  char* jobs = nullptr;    // job descriptors of the batched Gram-Schmidt stages
  size_t jobs_bytes = 0;
  double* Yd = nullptr;
  double* thd = nullptr;
  double* Xd = nullptr;
  size_t Xd_cap = 0;
  double* Wc = nullptr;       // n_pad x NBcap column-major (filtered block, unpacked)
  int32_t* colsel = nullptr;  // n_mesh x 8
  // stats
  kes_stats stats{};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_filter, ev_other;
  std::vector<cudaEvent_t> ev_pool;

  int n_mesh() const { return static_cast<int>(meshes.size()); }

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
  T* dalloc_n(int64_t count) {
    return static_cast<T*>(dalloc(static_cast<size_t>(count) * sizeof(T)));
  }
  template <typename T>
  T* dzero_n(int64_t count) {
    T* p = dalloc_n<T>(count);
    KES_CUDA(cudaMemsetAsync(p, 0, static_cast<size_t>(count) * sizeof(T), stream));
    return p;
  }

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
  void drop_graphs() {
    for (auto& g : graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }
};

namespace {

constexpr int kScal = 16;  // device scalars per mesh ahead of the Gram-Schmidt coefficients

void release(kes_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  c->drop_graphs();
  c->harvest_events();
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  while (!c->allocs.empty()) c->dfree(c->allocs.back().first);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

// --------------------------------------------------------------- transfers
// Caller block (n x nb column-major, host or device) -> row-major n_pad x NB block.
void block_in(kes_ctx* c, const double* src, int nb, int32_t mem, int NB, double* dst) {
  const size_t bytes = static_cast<size_t>(c->n) * nb * sizeof(double);
  KES_CUDA(cudaMemcpyAsync(c->tmp_user, src, bytes,
                           mem == KES_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
  launch_gather_rows(c->stream, c->tmp_user, c->n, nb, c->row_src, c->n, dst, NB, c->n_pad);
  KES_CHECK_LAUNCH();
}

// Row-major n_pad x NB block (first nb columns) -> caller block (n x nb column-major).
void block_out(kes_ctx* c, const double* src, int NB, int nb, double* dst, int32_t mem) {
  launch_scatter_rows(c->stream, src, NB, nb, c->row_src, c->n, c->tmp_user, c->n, c->n_pad);
  KES_CHECK_LAUNCH();
  KES_CUDA(cudaMemcpyAsync(dst, c->tmp_user, static_cast<size_t>(c->n) * nb * sizeof(double),
                           mem == KES_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
}

// --------------------------------------------------------------- filter
// Largest stable tau * omega of the context's stepper.
double cfl_bound(const kes_ctx* c) { return c->opts.stepper == KES_STEPPER_LEAPFROG4 ? 2.0 * std::sqrt(3.0) : 2.0; }

// Issues the fused steps of one filter application of an NB-column block on the context
// stream: stage_in -> stage_out (cpt = 0: F filtered blocks, every column with every
// weight table; cpt > 0: one block, column j with table min(j / cpt, F - 1)). steps <= L
// runs the first steps + 1 weights of the tables: alpha(t) of eq. (weightf) does not
// depend on T, so that is the filter of end time steps * tau.
int64_t issue_filter_steps(kes_ctx* c, int NB, bool fp64, int cpt, int steps) {
  const int64_t before = g_launches;
  const bool ho = c->opts.stepper == KES_STEPPER_LEAPFROG4;
  const int L = c->L, F = c->F;  // L: the tables' length (their stride is L + 1)
  const int64_t stride = c->n_pad * NB;
  if (fp64) {
    // in a context of the FP32 form the launch shape was tuned for the FP32 kernels:
    // the FP64 steps of the refinement take a fixed register-staged shape
    const SellDev A64 = c->step_A64();
    LaunchCfg cfg = c->cfg;
    if (c->opts.precision != KES_PREC_FP64) {
      cfg.variant = 3;
      cfg.grid_step = cfg.n_sm * step_blocks_per_sm(false, 3, cfg.block_step);
    }
    for (int s = 0; s < steps; ++s) {
      const bool first = s == 0, last = s == steps - 1;
      const double* x = s == 0 ? c->stage_in : c->U64[(s - 1) & 1];
      const double* prev = s <= 1 ? c->stage_in : c->U64[s & 1];
      double* out = c->U64[s & 1];
      const double* g = x;
      if (ho) {  // fourth order: the step gathers from v = u_n + A u_n / 12
        launch_stage4_f64(A64, cfg.n_sm, c->stream, NB, x, c->V64);
        g = c->V64;
      }
      if (NB == 1)
        launch_step_f64(A64, cfg, c->stream, first, x, g, prev, out, c->stage_out, stride, F, c->alpha64, L, s,
                        last, c->d_flag);
      else
        launch_step_blk_f64(A64, cfg, c->stream, NB, first, last, x, g, prev, out, c->stage_out, stride, F,
                            c->alpha64, L, s, cpt, c->d_flag);
    }
  } else {
    const SellDev A32 = c->step_A32();
    launch_init_f32(c->stream, c->A, NB, c->stage_in, c->U32[2], c->acc_s, c->acc_c, stride, F, c->alpha64, L, cpt);
    for (int s = 0; s < steps; ++s) {
      const bool first = s == 0, last = s == steps - 1;
      const float* x = s == 0 ? c->U32[2] : c->U32[(s - 1) & 1];
      const float* prev = s <= 1 ? c->U32[2] : c->U32[s & 1];
      float* out = c->U32[s & 1];
      const float* g = x;
      if (ho) {
        launch_stage4_f32(A32, c->cfg.n_sm, c->stream, NB, x, c->V32);
        g = c->V32;
      }
      if (NB == 1)
        launch_step_f32(A32, c->cfg, c->stream, first, last, x, g, prev, out, c->acc_s, c->acc_c, c->stage_out,
                        stride, F, c->alpha_hi, c->alpha_lo, L, s, c->d_flag);
      else
        launch_step_blk_f32(A32, c->cfg, c->stream, NB, first, last, x, g, prev, out, c->acc_s, c->acc_c,
                            c->stage_out, stride, F, c->alpha_hi, c->alpha_lo, L, s, cpt, c->d_flag);
    }
  }
  return g_launches - before;
}

// The FP64 step kernels in a context of the FP32 form (used by the FP64 refinement).
void ensure_fp64_state(kes_ctx* c) {
  if (!c->U64[0])
    for (int j = 0; j < 2; ++j) c->U64[j] = c->dzero_n<double>(c->n_pad * c->NBcap);
  if (!c->step64) {
    c->step64 = c->dzero_n<double>(c->nnz_pad);
    launch_scale_values(c->A, c->cfg, c->stream, c->tau2m64, c->step64, nullptr, nullptr, nullptr, c->fold64);
    KES_CHECK_LAUNCH();
  }
}

void run_filter(kes_ctx* c, int NB, bool fp64, int cpt = 0, int steps = 0) {
  if (cpt > 0 && NB < 2) throw KesError{KES_ERR_ARG};  // per-column tables live in the block kernels
  if (steps <= 0 || steps > c->L) steps = c->L;
  if (fp64) ensure_fp64_state(c);
  if (c->opts.stepper == KES_STEPPER_LEAPFROG4) {  // stage buffers before any graph captures them
    if (fp64 && !c->V64) c->V64 = c->dzero_n<double>(c->n_pad * c->NBcap);
    if (!fp64 && !c->V32) c->V32 = c->dzero_n<float>(c->n_pad * c->NBcap);
  }
  cudaEvent_t e0 = c->get_event(), e1 = c->get_event();
  KES_CUDA(cudaEventRecord(e0, c->stream));
  if (c->opts.use_graph) {
    if (c->g_F != c->F || c->g_L != c->L) {
      c->drop_graphs();
      c->g_F = c->F;
      c->g_L = c->L;
    }
    GraphEntry* ge = nullptr;
    for (auto& g : c->graphs)
      if (g.NB == NB && g.fp64 == fp64 && g.cpt == cpt && g.steps == steps) ge = &g;
    if (!ge) {
      cudaGraph_t graph;
      KES_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      const int64_t nodes = issue_filter_steps(c, NB, fp64, cpt, steps);
      cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
      g_launches -= nodes;  // captured, not launched
      KES_CUDA(ce);
      GraphEntry g;
      g.NB = NB;
      g.fp64 = fp64;
      g.cpt = cpt;
      g.steps = steps;
      g.nodes = nodes;
      ce = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      KES_CUDA(ce);
      c->graphs.push_back(g);
      ge = &c->graphs.back();
    }
    KES_CUDA(cudaGraphLaunch(ge->exec, c->stream));
    g_launches += ge->nodes;  // every node of the replayed graph is a kernel launch
  } else {
    issue_filter_steps(c, NB, fp64, cpt, steps);
    KES_CHECK_LAUNCH();
  }
  KES_CUDA(cudaEventRecord(e1, c->stream));
  c->ev_filter.emplace_back(e0, e1);
  c->stats.filter_calls += 1;
  c->stats.filter_steps += steps;
}

void ensure_stage_out(kes_ctx* c, int F) {
  if (c->stage_out_F >= F) return;
  const int64_t cnt = static_cast<int64_t>(F) * c->n_pad * c->NBcap;
  c->dfree(c->stage_out);
  c->stage_out = c->dzero_n<double>(cnt);
  if (c->opts.precision == KES_PREC_FP32) {
    c->dfree(c->acc_s);
    c->dfree(c->acc_c);
    c->acc_s = c->dzero_n<float>(cnt);
    c->acc_c = c->dzero_n<float>(cnt);
  }
  c->stage_out_F = F;
  c->drop_graphs();  // buffers moved: recapture
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
// A process is the Krylov iteration of one mesh on one interval (p = mesh * F + f).
void ensure_krylov(kes_ctx* c, int kmax, int F) {
  if (c->kcap >= kmax && c->kF >= F) return;
  for (double* p : {c->B, c->SB, c->Hd, c->partial, c->scal, c->Yd, c->thd, c->normd}) c->dfree(p);
  c->dfree(c->jobs);
  kmax = std::max(kmax, c->kcap);
  F = std::max(F, c->kF);
  const int64_t nproc = static_cast<int64_t>(c->n_mesh()) * F;
  c->kcap = kmax;
  c->kF = F;
  c->B = c->dzero_n<double>(static_cast<int64_t>(F) * kmax * c->n_pad);
  c->SB = c->dzero_n<double>(static_cast<int64_t>(F) * kmax * c->n_pad);
  c->Hd = c->dzero_n<double>(nproc * kmax * kmax);
  // partial sums: every process's inner products of one batched stage at once
  c->partial = c->dalloc_n<double>(nproc * kDotBlocks * (2 * kmax + 8));
  c->normd = c->dzero_n<double>(2 * nproc);
  // job descriptors of the batched Gram-Schmidt stages (see append_column)
  c->jobs_bytes = static_cast<size_t>(nproc) * (4 * sizeof(DotJob) + sizeof(GemvJob) + sizeof(ScaleJob)) +
                  static_cast<size_t>(2 * F * c->n_mesh()) * sizeof(double*) + 256;
  c->jobs = static_cast<char*>(c->dalloc(c->jobs_bytes));
  c->scal = c->dzero_n<double>(nproc * (2 * kmax + kScal));
  c->Yd = c->dalloc_n<double>(nproc * kmax * kmax);  // every process's selected Ritz vectors at once
  c->thd = c->dalloc_n<double>(nproc * kmax);
}

// Device scalars of process p (of mesh p outside the solver).
double* proc_scal(kes_ctx* c, int p) { return c->scal + static_cast<int64_t>(p) * (2 * c->kcap + kScal); }

// The slices of one mesh as a matrix of its own (columns stay global row indices).
SellDev mesh_sell(const kes_ctx* c, const MeshInfo& m) {
  SellDev a = c->A;
  a.slice_ptr = c->A.slice_ptr + m.slice_off;
  a.n_slices = m.n_slices;
  a.n = m.n;
  a.n_pad = m.n_pad;
  a.slice_mesh = nullptr;
  return a;
}

// Makes launch shape v of the single-vector step kernel current.
void select_variant(kes_ctx* c, int v) {
  const bool fp32 = c->opts.precision == KES_PREC_FP32;
  c->cfg.variant = v;
  c->cfg.grid_step = c->cfg.n_sm * step_blocks_per_sm(fp32, v, c->cfg.block_step);
}

// Times every launch shape of the step kernels on this matrix (a few steps on zeroed
// scratch state, CUDA events) and keeps the fastest. All shapes compute the same sums.
void tune_steps(kes_ctx* c) {
  const bool fp32 = c->opts.precision == KES_PREC_FP32;
  ensure_stage_out(c, 1);
  const int64_t na = static_cast<int64_t>(c->n_mesh()) * 8;
  double* a64 = c->dzero_n<double>(na);
  float* a32 = c->dzero_n<float>(na);
  cudaEvent_t e0 = c->get_event(), e1 = c->get_event();
  auto timed = [&](auto&& launch) {
    launch(3);
    float best = 3.0e38f;
    for (int rep = 0; rep < 3; ++rep) {
      KES_CUDA(cudaEventRecord(e0, c->stream));
      launch(16);
      KES_CUDA(cudaEventRecord(e1, c->stream));
      KES_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      KES_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      best = std::min(best, ms);
    }
    KES_CHECK_LAUNCH();
    return best;
  };
  // single-vector kernel
  int best = 0;
  float best_ms = 3.0e38f;
  for (int v = 0; v < step_variant_count(); ++v) {
    select_variant(c, v);
    const float ms = timed([&](int count) {
      for (int i = 0; i < count; ++i) {
        if (fp32)
          launch_step_f32(c->step_A32(), c->cfg, c->stream, false, false, c->U32[0], c->U32[0], c->U32[1], c->U32[1],
                          c->acc_s, c->acc_c, c->stage_out, c->n_pad, 1, a32, a32, 7, 1, c->d_flag);
        else
          launch_step_f64(c->step_A64(), c->cfg, c->stream, false, c->U64[0], c->U64[0], c->U64[1], c->U64[1],
                          c->stage_out, c->n_pad, 1, a64, 7, 1, false, c->d_flag);
      }
    });
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  select_variant(c, best);
  // block kernel at the context's block width
  if (c->NBcap > 1) {
    const int NB = c->NBcap;
    best = 0;
    best_ms = 3.0e38f;
    for (int v = 0; v < blk_variant_count(); ++v) {
      c->cfg.variant_blk = v;
      c->cfg.grid_blk = c->cfg.n_sm * blk_blocks_per_sm(fp32, NB, v, c->cfg.block_step);
      const float ms = timed([&](int count) {
        for (int i = 0; i < count; ++i) {
          if (fp32)
            launch_step_blk_f32(c->step_A32(), c->cfg, c->stream, NB, false, false, c->U32[0], c->U32[0], c->U32[1],
                                c->U32[1],
                                c->acc_s, c->acc_c, c->stage_out, c->n_pad * NB, 1, a32, a32, 7, 1, 0, c->d_flag);
          else
            launch_step_blk_f64(c->step_A64(), c->cfg, c->stream, NB, false, false, c->U64[0], c->U64[0], c->U64[1],
                                c->U64[1],
                                c->stage_out, c->n_pad * NB, 1, a64, 7, 1, 0, c->d_flag);
        }
      });
      if (ms < best_ms) {
        best_ms = ms;
        best = v;
      }
    }
    c->cfg.variant_blk = best;
    c->cfg.grid_blk = c->cfg.n_sm * blk_blocks_per_sm(fp32, NB, best, c->cfg.block_step);
  }
  c->ev_pool.push_back(e0);
  c->ev_pool.push_back(e1);
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

// Builds the block-diagonal device matrix and the per-row vectors of all meshes.
void build_context(kes_ctx* c, int nm, const int64_t* n, const int64_t* const* row_ptr, const int32_t* const* col,
                   const double* const* val, const double* const* m_diag) {
  std::vector<SellHost> sells(nm);
  int64_t row_off = 0, src_off = 0, slice_off = 0, nnz_pad = 0;
  for (int j = 0; j < nm; ++j) {  // inputs were validated by the caller
    MeshInfo mi;
    mi.n = n[j];
    mi.nnz = row_ptr[j][n[j]];
    double g = 0.0;
    for (int64_t i = 0; i < n[j]; ++i) {
      double s = 0.0;
      for (int64_t p = row_ptr[j][i]; p < row_ptr[j][i + 1]; ++p) s += std::fabs(val[j][p]);
      g = std::max(g, s / m_diag[j][i]);
    }
    mi.gershgorin = std::sqrt(g);
    sells[j] = build_sell(n[j], row_ptr[j], col[j], val[j], c->opts.sell_sigma);
    mi.n_slices = sells[j].n_slices;
    mi.n_pad = sells[j].n_slices * kSliceC;
    mi.row_off = row_off;
    mi.src_off = src_off;
    mi.slice_off = slice_off;
    row_off += mi.n_pad;
    src_off += mi.n;
    slice_off += mi.n_slices;
    nnz_pad += sells[j].nnz_pad;
    c->nnz += mi.nnz;
    c->meshes.push_back(mi);
  }
  c->n = src_off;
  c->n_pad = row_off;
  c->nnz_pad = nnz_pad;
  if (c->n >= (int64_t(1) << 31) || c->n_pad >= (int64_t(1) << 31)) throw KesError{KES_ERR_ARG};
  const int64_t n_slices = slice_off;
  // concatenate the slices; columns shift by the mesh's row offset
  std::vector<int64_t> sp(n_slices + 1);
  std::vector<int32_t> cols(nnz_pad);
  std::vector<double> vals(nnz_pad);
  std::vector<int32_t> smesh(n_slices), rsrc(c->n_pad, -1);
  std::vector<double> mp(c->n_pad, 0.0), minv(c->n_pad, 0.0);
  bool identity = nm == 1;
  int64_t at = 0;
  for (int j = 0; j < nm; ++j) {
    const MeshInfo& mi = c->meshes[j];
    const SellHost& sh = sells[j];
    for (int64_t s = 0; s < sh.n_slices; ++s) {
      sp[mi.slice_off + s] = at + sh.slice_ptr[s];
      smesh[mi.slice_off + s] = j;
    }
    for (int64_t e = 0; e < sh.nnz_pad; ++e) {
      cols[at + e] = static_cast<int32_t>(sh.col[e] + mi.row_off);
      vals[at + e] = sh.val[e];
    }
    at += sh.nnz_pad;
    for (int64_t i = 0; i < mi.n; ++i) {
      const int64_t o = sh.perm.empty() ? i : sh.perm[i];
      rsrc[mi.row_off + i] = static_cast<int32_t>(mi.src_off + o);
      if (mi.row_off + i != mi.src_off + o) identity = false;
      mp[mi.row_off + i] = m_diag[j][o];
      minv[mi.row_off + i] = 1.0 / m_diag[j][o];
    }
  }
  sp[n_slices] = at;
  sells.clear();
  // the leapfrog's 2 u_n folds into the diagonal of the FP64 step values when each row of a
  // mesh has an entry at its own column (a stored diagonal, or SELL padding of a short row,
  // which points at its row) among the first w of its slice; a slice of empty rows (w = 0)
  // has none. The padding rows past a mesh's last row need none: they gather only zeros,
  // read from no real row, and stay bounded (-u_(n-1)) with or without the 2 u_n.
  {
    bool diag = true;
    for (int64_t sl = 0; sl < n_slices && diag; ++sl) {
      const int64_t w = (sp[sl + 1] - sp[sl]) / kSliceC;
      for (int64_t l = 0; l < kSliceC && diag; ++l) {
        if (rsrc[sl * kSliceC + l] < 0) continue;  // padding row
        bool found = false;
        for (int64_t k = 0; k < w && !found; ++k) found = cols[sp[sl] + k * kSliceC + l] == sl * kSliceC + l;
        diag = found;
      }
    }
    c->diag_in_rows = diag;
  }
  // compact index for the step kernels: column - row as 16 bits when every entry allows it
  // (padding of a short row points at its own row: difference 0; padding rows past a mesh's
  // last row point at that row)
  std::vector<int16_t> dcol;
  if (c->opts.compact_cols) {
    dcol.resize(nnz_pad);
    bool fits = true;
    for (int64_t sl = 0; sl < n_slices && fits; ++sl)
      for (int64_t e = sp[sl]; e < sp[sl + 1]; ++e) {
        const int64_t row = sl * kSliceC + (e - sp[sl]) % kSliceC;
        const int64_t d = static_cast<int64_t>(cols[e]) - row;
        if (d < -32767 || d > 32767) {
          fits = false;
          break;
        }
        dcol[e] = static_cast<int16_t>(d);
      }
    if (!fits) dcol.clear();
  }
  int64_t* d_sp = c->dalloc_n<int64_t>(n_slices + 1);
  int32_t* d_col = c->dalloc_n<int32_t>(nnz_pad);
  double* d_val = c->dalloc_n<double>(nnz_pad);
  KES_CUDA(cudaMemcpyAsync(d_sp, sp.data(), (n_slices + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  KES_CUDA(cudaMemcpyAsync(d_col, cols.data(), nnz_pad * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  KES_CUDA(cudaMemcpyAsync(d_val, vals.data(), nnz_pad * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  c->A.n = c->n;
  c->A.n_pad = c->n_pad;
  c->A.n_slices = n_slices;
  c->A.slice_ptr = d_sp;
  c->A.col = d_col;
  if (!dcol.empty()) {
    int16_t* d_dcol = c->dalloc_n<int16_t>(nnz_pad);
    KES_CUDA(cudaMemcpyAsync(d_dcol, dcol.data(), nnz_pad * sizeof(int16_t), cudaMemcpyHostToDevice, c->stream));
    c->A.dcol = d_dcol;
    {
      // pair layout for the single-vector steps: entry k of lane l of slice s at
      // sp2[s] + 64 (k / 2) + 2 l + k % 2, odd widths padded with a zero entry per lane
      std::vector<int64_t> sp2(n_slices + 1, 0);
      for (int64_t sl = 0; sl < n_slices; ++sl) {
        const int64_t w = (sp[sl + 1] - sp[sl]) / kSliceC;
        sp2[sl + 1] = sp2[sl] + kSliceC * (w + (w & 1));
      }
      std::vector<int16_t> dcolp(sp2[n_slices], 0);
      for (int64_t sl = 0; sl < n_slices; ++sl)
        for (int64_t e = sp[sl]; e < sp[sl + 1]; ++e) {
          const int64_t k = (e - sp[sl]) / kSliceC, l = (e - sp[sl]) % kSliceC;
          dcolp[sp2[sl] + 64 * (k >> 1) + 2 * l + (k & 1)] = dcol[e];
        }
      c->nnz_pair = sp2[n_slices];
      int64_t* d_sp2 = c->dalloc_n<int64_t>(n_slices + 1);
      int16_t* d_dcolp = c->dalloc_n<int16_t>(c->nnz_pair);
      KES_CUDA(cudaMemcpyAsync(d_sp2, sp2.data(), (n_slices + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                               c->stream));
      KES_CUDA(cudaMemcpyAsync(d_dcolp, dcolp.data(), c->nnz_pair * sizeof(int16_t), cudaMemcpyHostToDevice,
                               c->stream));
      c->A.slice_ptr2 = d_sp2;
      c->A.dcolp = d_dcolp;
      c->sync();  // the host vectors go out of scope
    }
  }
  c->A.val64 = d_val;  // FP64 values are always kept: the Krylov basis needs S b_k in FP64
  if (c->opts.precision == KES_PREC_FP32) {
    std::vector<float> v32(vals.begin(), vals.end());
    float* d32 = c->dalloc_n<float>(nnz_pad);
    KES_CUDA(cudaMemcpyAsync(d32, v32.data(), nnz_pad * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    c->A.val32 = d32;
    c->sync();
  }
  if (nm > 1) {
    c->slice_mesh = c->dalloc_n<int32_t>(n_slices);
    KES_CUDA(cudaMemcpyAsync(c->slice_mesh, smesh.data(), n_slices * sizeof(int32_t), cudaMemcpyHostToDevice,
                             c->stream));
    c->A.slice_mesh = c->slice_mesh;
  }
  if (!identity) {
    c->row_src = c->dalloc_n<int32_t>(c->n_pad);
    KES_CUDA(
        cudaMemcpyAsync(c->row_src, rsrc.data(), c->n_pad * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  }
  c->m64 = c->dalloc_n<double>(c->n_pad);
  c->minv64 = c->dalloc_n<double>(c->n_pad);
  KES_CUDA(cudaMemcpyAsync(c->m64, mp.data(), c->n_pad * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  KES_CUDA(cudaMemcpyAsync(c->minv64, minv.data(), c->n_pad * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  c->sync();
}

kes_status create_impl(kes_ctx** out, int32_t nm, const int64_t* n, const int64_t* const* row_ptr,
                       const int32_t* const* col, const double* const* val, const double* const* m_diag,
                       const kes_opts* opts) {
  if (!out) return KES_ERR_ARG;
  *out = nullptr;
  if (nm < 1 || !n || !row_ptr || !col || !val || !m_diag) return KES_ERR_ARG;
  kes_ctx* c = nullptr;
  kes_status st = guarded([&]() -> kes_status {
    c = new kes_ctx();
    if (opts) c->opts = *opts;
    else kes_opts_default(&c->opts);
    if (c->opts.precision != KES_PREC_FP64 && c->opts.precision != KES_PREC_FP32) throw KesError{KES_ERR_ARG};
    if (c->opts.sell_sigma < 1) c->opts.sell_sigma = 1;
    if (c->opts.block_b < 1) c->opts.block_b = 1;
    if (c->opts.block_b > 8) throw KesError{KES_ERR_UNSUPPORTED};
    if ((c->opts.dev_alloc == nullptr) != (c->opts.dev_free == nullptr)) throw KesError{KES_ERR_ARG};
    if (c->opts.step_variant < 0 || c->opts.step_variant >= step_variant_count()) throw KesError{KES_ERR_ARG};
    if (c->opts.blk_variant < 0 || c->opts.blk_variant >= blk_variant_count()) throw KesError{KES_ERR_ARG};
    if (c->opts.stepper != KES_STEPPER_LEAPFROG && c->opts.stepper != KES_STEPPER_LEAPFROG4)
      throw KesError{KES_ERR_ARG};
    // host-side validation first: a bad input never reaches the GPU
    for (int j = 0; j < nm; ++j) {
      if (!row_ptr[j] || !col[j] || !val[j] || !m_diag[j]) throw KesError{KES_ERR_ARG};
      validate_csr(n[j], row_ptr[j], col[j], val[j], m_diag[j]);
    }
    c->NBcap = nb_for(c->opts.block_b);
    KES_CUDA(cudaGetDevice(&c->device));
    int n_sm = 0;
    KES_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device));
    if (c->opts.stream) {
      c->stream = static_cast<cudaStream_t>(c->opts.stream);
    } else {
      KES_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    build_context(c, nm, n, row_ptr, col, val, m_diag);
    c->fold64 = c->diag_in_rows && c->opts.stepper == KES_STEPPER_LEAPFROG;
    const int64_t np = c->n_pad, nb = c->NBcap;
    c->tau2m64 = c->dzero_n<double>(np);
    if (c->opts.precision == KES_PREC_FP32) {
      c->step32 = c->dzero_n<float>(c->nnz_pad);
      if (c->A.slice_ptr2) c->step32p = c->dzero_n<float>(c->nnz_pair);  // padding stays zero
      for (int j = 0; j < 3; ++j) c->U32[j] = c->dzero_n<float>(np * nb);
    } else {
      c->step64 = c->dzero_n<double>(c->nnz_pad);
      if (c->A.slice_ptr2 && c->fold64) c->step64p = c->dzero_n<double>(c->nnz_pair);  // padding stays zero
      for (int j = 0; j < 2; ++j) c->U64[j] = c->dzero_n<double>(np * nb);
    }
    c->stage_in = c->dzero_n<double>(np * nb);
    c->tmp_user = c->dzero_n<double>(c->n * nb);
    c->Wc = c->dzero_n<double>(np * nb);
    c->colsel = c->dalloc_n<int32_t>(static_cast<int64_t>(nm) * 8);
    c->d_flag = c->dzero_n<int>(4);
    // grid-stride launch shapes: one full wave of resident 256-thread blocks
    const bool fp32 = c->opts.precision == KES_PREC_FP32;
    c->cfg.n_sm = n_sm;
    c->cfg.block_step = 256;
    select_variant(c, c->opts.step_variant);
    c->cfg.variant_blk = c->opts.blk_variant;
    c->cfg.grid_blk =
        n_sm * blk_blocks_per_sm(fp32, c->NBcap > 1 ? c->NBcap : 2, c->opts.blk_variant, c->cfg.block_step);
    if (c->opts.autotune) tune_steps(c);
    c->sync();
    c->stats.bytes_per_step = kes_step_bytes(c, 1, 1);
    c->stats.step_variant = c->cfg.variant;
    c->stats.step_grid = c->cfg.grid_step;
    c->stats.blk_variant = c->NBcap > 1 ? c->cfg.variant_blk : -1;
    c->stats.blk_grid = c->NBcap > 1 ? c->cfg.grid_blk : 0;
    return KES_OK;
  });
  if (st != KES_OK) {
    release(c);
    return st;
  }
  *out = c;
  return KES_OK;
}

// Installs F weight tables per mesh (alpha: [n_mesh][F][L+1], or null: the indicator
// weights of eq. (weightf) for [wmin, wmax]); [wmin, wmax] is also the interval in which
// the solver accepts Ritz pairs.
kes_status set_weights_impl(kes_ctx* c, int32_t F, const double* alpha, const double* wmin, const double* wmax,
                            const double* tau, int32_t L) {
  const int nm = c->n_mesh();
  for (int j = 0; j < nm; ++j) {
    if (!(tau[j] > 0.0) || !std::isfinite(tau[j])) return KES_ERR_ARG;
    for (int f = 0; f < F; ++f) {
      const double a = wmin[j * F + f], b = wmax[j * F + f];
      if (!(a >= 0.0) || !(b > a) || !std::isfinite(b)) return KES_ERR_ARG;
    }
    if (c->meshes[j].omega_est > 0.0 && tau[j] * c->meshes[j].omega_est >= cfl_bound(c)) return KES_ERR_UNSTABLE;
  }
  const size_t need = static_cast<size_t>(nm) * F * (L + 1);
  if (alpha)
    for (size_t i = 0; i < need; ++i)
      if (!std::isfinite(alpha[i])) return KES_ERR_ARG;
  return guarded([&]() -> kes_status {
    std::vector<double> a64(need, 0.0);
    if (alpha) {
      std::memcpy(a64.data(), alpha, need * sizeof(double));
    } else {
      for (int j = 0; j < nm; ++j)
        for (int f = 0; f < F; ++f)
          alpha_table(wmin[j * F + f], wmax[j * F + f], tau[j], L,
                      a64.data() + (static_cast<size_t>(j) * F + f) * (L + 1));
    }
    c->sync();
    if (need > c->alpha_cap) {
      c->dfree(c->alpha64);
      c->dfree(c->alpha_hi);
      c->dfree(c->alpha_lo);
      c->alpha64 = c->dalloc_n<double>(need);
      c->alpha_hi = c->dalloc_n<float>(need);
      c->alpha_lo = c->dalloc_n<float>(need);
      c->alpha_cap = need;
      c->drop_graphs();
    }
    std::vector<float> hi(need), lo(need);
    for (size_t i = 0; i < need; ++i) {
      hi[i] = static_cast<float>(a64[i]);
      lo[i] = static_cast<float>(a64[i] - static_cast<double>(hi[i]));
    }
    KES_CUDA(cudaMemcpyAsync(c->alpha64, a64.data(), need * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    KES_CUDA(cudaMemcpyAsync(c->alpha_hi, hi.data(), need * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    KES_CUDA(cudaMemcpyAsync(c->alpha_lo, lo.data(), need * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    // tau^2 / m with each mesh's tau, in the padded (permuted) order
    std::vector<double> m(c->n_pad);
    KES_CUDA(cudaMemcpyAsync(m.data(), c->m64, c->n_pad * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    c->sync();
    std::vector<double> t2m(c->n_pad, 0.0);
    for (int j = 0; j < nm; ++j) {
      const MeshInfo& mi = c->meshes[j];
      for (int64_t i = 0; i < mi.n; ++i) t2m[mi.row_off + i] = tau[j] * tau[j] / m[mi.row_off + i];
    }
    KES_CUDA(cudaMemcpyAsync(c->tau2m64, t2m.data(), c->n_pad * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    // step values A = -tau^2 M^{-1} S (the FP32 ones rounded once from the FP64 product)
    if (c->step64 || c->step32)
      launch_scale_values(c->A, c->cfg, c->stream, c->tau2m64, c->step64, c->step32, c->step64p, c->step32p,
                          c->fold64);
    KES_CHECK_LAUNCH();
    ensure_stage_out(c, F);
    c->sync();
    c->F = F;
    c->L = L;
    for (int j = 0; j < nm; ++j) {
      c->meshes[j].tau = tau[j];
      c->meshes[j].wmin.assign(wmin + j * F, wmin + (j + 1) * F);
      c->meshes[j].wmax.assign(wmax + j * F, wmax + (j + 1) * F);
    }
    c->filter_set = true;
    return KES_OK;
  });
}

kes_status omega_impl(kes_ctx* c, int32_t iters, const double* v0, double* omega, double* gersh) {
  LaunchCount lc(&c->stats);
  return guarded([&]() -> kes_status {
    const int nm = c->n_mesh();
    ensure_krylov(c, 2, 1);
    double* v = c->B;  // scratch n_pad vectors
    double* w = c->SB;
    cudaStream_t s = c->stream;
    block_in(c, v0, 1, KES_MEM_HOST, 1, w);
    for (int j = 0; j < nm; ++j) {
      const MeshInfo& mi = c->meshes[j];
      double* sc = proc_scal(c, j);
      launch_mdot(s, w + mi.row_off, 0, 1, w + mi.row_off, nullptr, mi.n_pad, c->partial, sc);
      launch_scale_rsqrt(s, w + mi.row_off, sc, v + mi.row_off, nullptr, mi.n_pad);
    }
    for (int it = 0; it < iters; ++it) {
      launch_spmv_f64(c->A, c->cfg, s, v, c->minv64, w);
      for (int j = 0; j < nm; ++j) {
        const MeshInfo& mi = c->meshes[j];
        double* sc = proc_scal(c, j);
        launch_mdot(s, w + mi.row_off, 0, 1, w + mi.row_off, nullptr, mi.n_pad, c->partial, sc);
        launch_scale_rsqrt(s, w + mi.row_off, sc, v + mi.row_off, nullptr, mi.n_pad);
      }
    }
    launch_spmv_f64(c->A, c->cfg, s, v, nullptr, w);
    std::vector<double> h(2 * nm);
    for (int j = 0; j < nm; ++j) {
      const MeshInfo& mi = c->meshes[j];
      double* sc = proc_scal(c, j);
      launch_mdot(s, v + mi.row_off, 0, 1, w + mi.row_off, nullptr, mi.n_pad, c->partial, sc);  // v^T S v
      launch_mdot(s, v + mi.row_off, 0, 1, v + mi.row_off, c->m64 + mi.row_off, mi.n_pad, c->partial,
                  sc + 1);  // v^T M v
      KES_CUDA(cudaMemcpyAsync(&h[2 * j], sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    KES_CHECK_LAUNCH();
    c->sync();
    for (int j = 0; j < nm; ++j) {
      omega[j] = std::sqrt(std::max(h[2 * j], 0.0) / h[2 * j + 1]);
      c->meshes[j].omega_est = omega[j];
      if (gersh) gersh[j] = c->meshes[j].gershgorin;
    }
    return KES_OK;
  });
}

// ------------------------------------------------------------------ block Krylov solver
struct MeshSolve {
  int k = 0;            // basis vectors
  bool done = false;    // no further blocks for this process
  bool breakdown = false;
  int kproj = -1;       // basis size at the last projection
  std::vector<double> last_theta, last_rel;
  std::vector<double> acc_theta, acc_rel, acc_abs, acc_Y;
};

// Sets each job's first block of a batched launch (prefix sums in job order) and returns
// the launch's total blocks.
inline int64_t job_blocks(const DotJob& j) { return dot_job_blocks(j); }
inline int64_t job_blocks(const GemvJob& j) { return gemv_job_blocks(j); }
template <typename J>
int64_t first_blocks(std::vector<J>& jobs) {
  int64_t total = 0;
  for (J& j : jobs) {
    j.first = total;
    total += job_blocks(j);
  }
  return total;
}

template <typename T>
T* hdup(const std::vector<T>& v) {
  T* d = static_cast<T*>(std::malloc(std::max<size_t>(1, v.size()) * sizeof(T)));
  if (!d) throw std::bad_alloc();
  if (!v.empty()) std::memcpy(d, v.data(), v.size() * sizeof(T));
  return d;
}


// The block solver over every mesh and interval of the context. Process p = mesh * F + f
// is the block Krylov iteration of mesh p / F on interval f from start columns
// f * g .. f * g + g - 1 (g = b / F), with its own basis, Gram-Schmidt scalars and
// projected matrix; the processes share only the b-column trajectory of each block step.
// X0 (p0 caller vectors, n_total x p0 column-major) selects the fixed-dimension mode: no
// Krylov phase; refine_sweeps sweeps of X <- C X, M-orthonormalisation and Rayleigh-Ritz
// from X0, every Ritz vector fed back (the FEAST-like use of the filter in Sec. 4).
kes_status block_solve_impl(kes_ctx* c, const double* R0, int b, int32_t mem, const kes_solve_opts& so,
                            kes_result** out, const double* X0 = nullptr, int p0 = 0) {
  const int nm = c->n_mesh();
  const int F = c->F;
  const int P = nm * F;
  const int g = b / F;                // columns per process
  const int cpt = F > 1 ? g : 0;      // column j of a block takes weight table j / g
  const int kmax = so.kmax;
  const int NB = nb_for(b);
  std::vector<MeshSolve> ms(P);
  std::vector<kes_result*> res(nm, nullptr);
  for (int j = 0; j < nm; ++j) {
    res[j] = static_cast<kes_result*>(std::calloc(1, sizeof(kes_result)));
    if (!res[j]) {
      for (auto* r : res) kes_result_free(r);
      return KES_ERR_OOM;
    }
  }
  const auto t_start = std::chrono::steady_clock::now();
  LaunchCount lc(&c->stats);
  kes_status st = guarded([&]() -> kes_status {
    ensure_krylov(c, kmax, F);
    const int64_t np = c->n_pad;
    const int64_t kc = c->kcap;
    cudaStream_t s = c->stream;
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
    auto mesh_of = [&](int p) -> const MeshInfo& { return c->meshes[p / F]; };
    // column 0 of process p's basis over all rows (SpMV input) and on its mesh's rows
    auto Bfull = [&](int p) { return c->B + (p % F) * kc * np; };
    auto Bp = [&](int p) { return Bfull(p) + mesh_of(p).row_off; };
    auto SBp = [&](int p) { return c->SB + (p % F) * kc * np + mesh_of(p).row_off; };
    auto Hcol = [&](int p, int k) { return c->Hd + (static_cast<int64_t>(p) * kc + k) * kc; };
    // process that owns column jj of a block of mesh j (-1: a padding column)
    auto owner = [&](int j, int jj) {
      const int f = F > 1 ? jj / g : 0;
      return f < F ? j * F + f : -1;
    };

    // Orthogonalise column jj of Wc against the basis of the process that owns it on
    // each mesh (two classical passes in the M-inner product) and append the vectors
    // that are not dependent (Algorithm 2.5).
    std::vector<char> want(P, 1);  // processes taking part in the current block step
    auto append_column = [&](int jj) {
      std::vector<char> added(P, 0);
      std::vector<int> act;  // processes that take column jj
      for (int j = 0; j < nm; ++j) {
        const int p = owner(j, jj);
        if (p < 0 || !want[p] || ms[p].done || ms[p].k >= kmax) continue;
        act.push_back(p);
      }
      if (act.empty()) return added;
      const int na = static_cast<int>(act.size());
      // phase 1, one launch per stage for all of them: ||w||_M^2, two passes of
      // h = B^T M w and w -= B h, ||w||_M^2 again
      std::vector<DotJob> nb_jobs(na), na_jobs(na), h_jobs;
      std::vector<GemvJob> g_jobs;
      int max_k = 0;
      int64_t poff = 0, poff_h = 0;
      for (int i = 0; i < na; ++i) {
        const int p = act[i];
        const MeshInfo& mi = mesh_of(p);
        double* w = c->Wc + static_cast<int64_t>(jj) * np + mi.row_off;
        const double* mj = c->m64 + mi.row_off;
        const int nblk = dot_blocks(mi.n_pad), gblk = gemv_blocks(mi.n_pad);
        nb_jobs[i] = DotJob{w, w, mj, c->normd + 2 * p, mi.n_pad, 0, poff, 0, 1, nblk};
        na_jobs[i] = DotJob{w, w, mj, c->normd + 2 * p + 1, mi.n_pad, 0, poff, 0, 1, nblk};
        poff += nblk;
        const int k = ms[p].k;
        if (k > 0) {
          h_jobs.push_back(DotJob{Bp(p), w, mj, proc_scal(c, p) + kScal, mi.n_pad, np, poff_h, 0, k, nblk});
          g_jobs.push_back(GemvJob{w, Bp(p), proc_scal(c, p) + kScal, mi.n_pad, np, 0, k, gblk});
          poff_h += static_cast<int64_t>(k) * nblk;
          max_k = std::max(max_k, k);
        }
      }
      const int nh = static_cast<int>(h_jobs.size());
      const int64_t nb_blocks = first_blocks(nb_jobs), na_blocks = first_blocks(na_jobs);
      const int64_t h_blocks = first_blocks(h_jobs), g_blocks = first_blocks(g_jobs);
      char* jb = c->jobs;
      DotJob* d_nb = reinterpret_cast<DotJob*>(jb);
      DotJob* d_na = d_nb + P;
      DotJob* d_h = d_na + P;
      GemvJob* d_g = reinterpret_cast<GemvJob*>(d_h + P);
      cudaEvent_t ev = other_begin();
      KES_CUDA(cudaMemcpyAsync(d_nb, nb_jobs.data(), na * sizeof(DotJob), cudaMemcpyHostToDevice, s));
      KES_CUDA(cudaMemcpyAsync(d_na, na_jobs.data(), na * sizeof(DotJob), cudaMemcpyHostToDevice, s));
      if (nh > 0) {
        KES_CUDA(cudaMemcpyAsync(d_h, h_jobs.data(), nh * sizeof(DotJob), cudaMemcpyHostToDevice, s));
        KES_CUDA(cudaMemcpyAsync(d_g, g_jobs.data(), nh * sizeof(GemvJob), cudaMemcpyHostToDevice, s));
      }
      launch_mdot_jobs(s, d_nb, na, 1, nb_blocks, c->partial);  // ||w||_M^2 before
      for (int pass = 0; pass < 2 && nh > 0; ++pass) {
        launch_mdot_jobs(s, d_h, nh, max_k, h_blocks, c->partial);  // h = B^T M w
        launch_gemv_sub_jobs(s, d_g, nh, max_k, g_blocks);          // w -= B h
      }
      launch_mdot_jobs(s, d_na, na, 1, na_blocks, c->partial);  // ||w||_M^2 after
      KES_CHECK_LAUNCH();
      std::vector<double> nrm(2 * P, 0.0);
      KES_CUDA(cudaMemcpyAsync(nrm.data(), c->normd, 2 * P * sizeof(double), cudaMemcpyDeviceToHost, s));
      int flag = 0;
      KES_CUDA(cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      other_end(ev);
      c->sync();
      if (flag) {
        KES_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
        throw KesError{KES_ERR_UNSTABLE};
      }
      // phase 2 for the vectors that are not dependent: b_k = w / ||w||_M, S b_k (one
      // launch per interval over all meshes), the new column b_i^T S b_k of H
      std::vector<ScaleJob> s_jobs;
      std::vector<DotJob> c_jobs;
      std::vector<const double*> x_of(static_cast<size_t>(F) * nm, nullptr);
      std::vector<double*> y_of(static_cast<size_t>(F) * nm, nullptr);
      int max_k1 = 0, max_sblk = 1;
      poff = 0;
      for (int i = 0; i < na; ++i) {
        const int p = act[i];
        if (!(std::sqrt(nrm[2 * p + 1]) > 1e-10 * std::sqrt(nrm[2 * p]))) continue;  // dependent vector
        const MeshInfo& mi = mesh_of(p);
        const int k = ms[p].k;
        double* w = c->Wc + static_cast<int64_t>(jj) * np + mi.row_off;
        double* sbk = SBp(p) + k * np;
        const int nblk = dot_blocks(mi.n_pad);
        s_jobs.push_back(ScaleJob{w, c->normd + 2 * p + 1, Bp(p) + k * np, mi.n_pad});
        max_sblk = std::max(max_sblk, gemv_blocks(mi.n_pad));
        x_of[static_cast<size_t>(p % F) * nm + p / F] = Bfull(p) + k * np;
        y_of[static_cast<size_t>(p % F) * nm + p / F] = c->SB + (p % F) * kc * np + k * np;
        c_jobs.push_back(DotJob{Bp(p), sbk, nullptr, Hcol(p, k), mi.n_pad, np, poff, 0, k + 1, nblk});
        poff += static_cast<int64_t>(k + 1) * nblk;
        max_k1 = std::max(max_k1, k + 1);
        ms[p].k = k + 1;
        added[p] = 1;
      }
      const int ns = static_cast<int>(s_jobs.size());
      const int64_t c_blocks = first_blocks(c_jobs);
      if (ns > 0) {
        ev = other_begin();
        ScaleJob* d_s = reinterpret_cast<ScaleJob*>(d_g + P);
        DotJob* d_c = reinterpret_cast<DotJob*>(d_s + P);
        char* ptrs = reinterpret_cast<char*>(d_c + P);  // x_of, then y_of, F * nm pointers each
        const double** d_x = reinterpret_cast<const double**>(ptrs);
        double** d_y = reinterpret_cast<double**>(ptrs + static_cast<size_t>(F) * nm * sizeof(double*));
        KES_CUDA(cudaMemcpyAsync(d_s, s_jobs.data(), ns * sizeof(ScaleJob), cudaMemcpyHostToDevice, s));
        KES_CUDA(cudaMemcpyAsync(d_c, c_jobs.data(), ns * sizeof(DotJob), cudaMemcpyHostToDevice, s));
        KES_CUDA(cudaMemcpyAsync(d_x, x_of.data(), x_of.size() * sizeof(double*), cudaMemcpyHostToDevice, s));
        KES_CUDA(cudaMemcpyAsync(d_y, y_of.data(), y_of.size() * sizeof(double*), cudaMemcpyHostToDevice, s));
        launch_scale_jobs(s, d_s, ns, max_sblk);
        for (int f = 0; f < F; ++f) {
          bool any = false;
          for (int j = 0; j < nm; ++j) any |= x_of[static_cast<size_t>(f) * nm + j] != nullptr;
          if (any) launch_spmv_f64_meshes(c->A, c->cfg, s, d_x + static_cast<size_t>(f) * nm,
                                          d_y + static_cast<size_t>(f) * nm);
        }
        launch_mdot_jobs(s, d_c, ns, max_k1, c_blocks, c->partial);
        KES_CHECK_LAUNCH();
        other_end(ev);
      }
      return added;
    };

    // The projected matrix of process p mirrored into a full kk x kk array and its
    // eigenpairs (theta ascending, clamped at 0).
    auto projected_eig = [&](int p, std::vector<double>& theta, std::vector<double>& Y) {
      const int kk = ms[p].k;
      std::vector<double> Hh(static_cast<size_t>(kk) * kk, 0.0);
      KES_CUDA(cudaMemcpy2DAsync(Hh.data(), kk * sizeof(double), Hcol(p, 0), kc * sizeof(double),
                                 kk * sizeof(double), kk, cudaMemcpyDeviceToHost, s));
      c->sync();
      // column i holds rows 0..i (upper triangle); mirror it into the lower triangle
      for (int i = 0; i < kk; ++i)
        for (int r = i + 1; r < kk; ++r) Hh[static_cast<size_t>(i) * kk + r] = Hh[static_cast<size_t>(r) * kk + i];
      theta.assign(kk, 0.0);
      Y.assign(static_cast<size_t>(kk) * kk, 0.0);
      if (!sym_eig(kk, Hh.data(), theta.data(), Y.data())) throw KesError{KES_ERR_CUDA};
      for (double& t : theta) t = std::max(t, 0.0);
    };

    // Rayleigh-Ritz (eq. projevp) and the residual acceptance (eq. res) of several
    // processes at once: their projected matrices come back with one synchronisation,
    // the small eigenproblems are solved on host threads, and the residual kernels run
    // back to back before one more synchronisation.
    auto project_many = [&](const std::vector<int>& ps) {
      const int np_ = static_cast<int>(ps.size());
      if (np_ == 0) return;
      std::vector<std::vector<double>> Hs(np_), th(np_), Ys(np_);
      for (int i = 0; i < np_; ++i) {
        const int kk = ms[ps[i]].k;
        Hs[i].assign(static_cast<size_t>(kk) * kk, 0.0);
        if (kk > 0)
          KES_CUDA(cudaMemcpy2DAsync(Hs[i].data(), kk * sizeof(double), Hcol(ps[i], 0), kc * sizeof(double),
                                     kk * sizeof(double), kk, cudaMemcpyDeviceToHost, s));
      }
      c->sync();
      std::atomic<int> next{0};
      std::atomic<bool> failed{false};
      auto worker = [&]() {
        for (int i = next++; i < np_; i = next++) {
          const int kk = ms[ps[i]].k;
          std::vector<double>& H = Hs[i];
          // column i holds rows 0..i (upper triangle); mirror it into the lower triangle
          for (int a = 0; a < kk; ++a)
            for (int r = a + 1; r < kk; ++r) H[static_cast<size_t>(a) * kk + r] = H[static_cast<size_t>(r) * kk + a];
          th[i].assign(kk, 0.0);
          Ys[i].assign(static_cast<size_t>(kk) * kk, 0.0);
          if (!sym_eig(kk, H.data(), th[i].data(), Ys[i].data())) failed = true;
          for (double& t : th[i]) t = std::max(t, 0.0);
        }
      };
      const int hw = static_cast<int>(std::thread::hardware_concurrency());
      const int nt = std::min(np_, std::max(1, std::min(hw, 16)));
      std::vector<std::thread> pool;
      for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
      worker();
      for (auto& t : pool) t.join();
      if (failed) throw KesError{KES_ERR_CUDA};
      std::vector<std::vector<int>> inside(np_);
      std::vector<std::vector<double>> Ysel(np_), thsel(np_), rr(np_);
      cudaEvent_t ev = other_begin();
      int64_t yo = 0, to = 0;
      for (int i = 0; i < np_; ++i) {
        const int p = ps[i];
        MeshSolve& m = ms[p];
        const MeshInfo& mi = mesh_of(p);
        const int kk = m.k;
        m.kproj = kk;
        const double wmin = mi.wmin[p % F], wmax = mi.wmax[p % F];
        for (int q = 0; q < kk; ++q) {
          const double om = std::sqrt(th[i][q]);
          if (om >= wmin && om <= wmax) inside[i].push_back(q);
        }
        const int np_in = static_cast<int>(inside[i].size());
        m.last_theta = th[i];
        m.last_rel.assign(kk, std::numeric_limits<double>::quiet_NaN());
        m.acc_theta.clear();
        m.acc_rel.clear();
        m.acc_abs.clear();
        m.acc_Y.clear();
        if (np_in == 0) continue;
        Ysel[i].resize(static_cast<size_t>(kk) * np_in);
        thsel[i].resize(np_in);
        for (int q = 0; q < np_in; ++q) {
          thsel[i][q] = th[i][inside[i][q]];
          std::memcpy(&Ysel[i][static_cast<size_t>(q) * kk], &Ys[i][static_cast<size_t>(inside[i][q]) * kk],
                      kk * sizeof(double));
        }
        KES_CUDA(cudaMemcpyAsync(c->Yd + yo, Ysel[i].data(), Ysel[i].size() * sizeof(double), cudaMemcpyHostToDevice,
                                 s));
        KES_CUDA(cudaMemcpyAsync(c->thd + to, thsel[i].data(), np_in * sizeof(double), cudaMemcpyHostToDevice, s));
        double* sc = proc_scal(c, p);
        launch_ritz_residual(s, Bp(p), SBp(p), np, kk, c->Yd + yo, c->thd + to, np_in, c->m64 + mi.row_off,
                             mi.n_pad, c->partial, sc + kScal);
        KES_CHECK_LAUNCH();
        rr[i].resize(2 * np_in);
        KES_CUDA(cudaMemcpyAsync(rr[i].data(), sc + kScal, 2 * np_in * sizeof(double), cudaMemcpyDeviceToHost, s));
        yo += static_cast<int64_t>(kk) * np_in;
        to += np_in;
      }
      other_end(ev);
      c->sync();
      for (int i = 0; i < np_; ++i) {
        MeshSolve& m = ms[ps[i]];
        const int kk = m.k;
        const int np_in = static_cast<int>(inside[i].size());
        for (int q = 0; q < np_in; ++q) {
          const double a = std::sqrt(std::max(rr[i][q], 0.0));
          const double den = thsel[i][q] * std::sqrt(std::max(rr[i][np_in + q], 0.0));
          const double rel = den > 0.0 ? a / den : std::numeric_limits<double>::infinity();
          m.last_rel[inside[i][q]] = rel;
          if (rel <= so.tol) {
            m.acc_theta.push_back(thsel[i][q]);
            m.acc_rel.push_back(rel);
            m.acc_abs.push_back(a);
            m.acc_Y.insert(m.acc_Y.end(), Ysel[i].begin() + static_cast<size_t>(q) * kk,
                           Ysel[i].begin() + static_cast<size_t>(q + 1) * kk);
          }
        }
      }
    };

    // a mesh that asked for n_wanted pairs stops once its intervals hold that many
    auto check_wanted = [&]() {
      if (so.n_wanted <= 0) return;
      for (int j = 0; j < nm; ++j) {
        int got = 0;
        for (int f = 0; f < F; ++f) got += static_cast<int>(ms[j * F + f].acc_theta.size());
        if (got >= so.n_wanted)
          for (int f = 0; f < F; ++f) ms[j * F + f].done = true;
      }
    };

    int64_t steps = 0;
    // start block: the g start vectors of each process, M-orthonormalised in order
    if (!X0) {
      cudaEvent_t ev = other_begin();
      block_in(c, R0, b, mem, NB, c->stage_in);
      launch_unpack_block(s, c->stage_in, NB, c->Wc, np);
      KES_CHECK_LAUNCH();
      other_end(ev);
      for (int jj = 0; jj < b; ++jj) append_column(jj);
      for (int p = 0; p < P; ++p)
        if (ms[p].k == 0) ms[p].done = ms[p].breakdown = true;
    }
    std::vector<int> next_check(P, so.check_every);
    std::vector<int32_t> colsel(static_cast<size_t>(nm) * NB, -1);
    for (; !X0;) {
      bool any = false;
      std::fill(colsel.begin(), colsel.end(), -1);
      for (int p = 0; p < P; ++p) {
        MeshSolve& m = ms[p];
        if (m.done || m.k >= kmax) continue;
        any = true;
        // filter the g newest basis vectors of each process (Algorithm 2.5 filters the newest one)
        const int j = p / F, f = p % F;
        for (int i = 0; i < g; ++i) {
          const int col = m.k - g + i;
          colsel[j * NB + f * g + i] = col >= 0 ? static_cast<int32_t>(f * kc + col) : -1;
        }
      }
      if (!any) break;
      KES_CUDA(cudaMemcpyAsync(c->colsel, colsel.data(), colsel.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
      launch_pack_basis(s, c->B, np, c->colsel, c->slice_mesh, c->stage_in, NB, np);
      KES_CHECK_LAUNCH();
      run_filter(c, NB, c->opts.precision == KES_PREC_FP64, cpt);  // stage_in -> stage_out
      steps += c->L;
      launch_unpack_block(s, c->stage_out, NB, c->Wc, np);
      KES_CHECK_LAUNCH();
      std::vector<int> added(P, 0);
      for (int jj = 0; jj < b; ++jj) {
        std::vector<char> a = append_column(jj);
        for (int p = 0; p < P; ++p) added[p] += a[p];
      }
      std::vector<int> due;
      for (int p = 0; p < P; ++p) {
        MeshSolve& m = ms[p];
        if (m.done) continue;
        if (added[p] == 0 && m.k < kmax) {  // the whole block was dependent: invariant subspace
          m.done = m.breakdown = true;
          continue;
        }
        if (m.k >= next_check[p] && m.k < kmax) {
          while (next_check[p] <= m.k) next_check[p] += so.check_every;
          due.push_back(p);
        }
      }
      project_many(due);
      check_wanted();
    }
    if (!X0) {
      std::vector<int> due;
      for (int p = 0; p < P; ++p)
        if (ms[p].kproj != ms[p].k) due.push_back(p);
      project_many(due);
    }

    // FP64 refinement: sweeps of filtered subspace iteration on the in-interval Ritz
    // vectors of each process (Sec. 4 mentions fixed-dimension, FEAST-like use of the
    // filter): X <- C X with the FP64 step kernels, M-orthonormalise, Rayleigh-Ritz,
    // residuals. With F intervals the columns of a refinement block are grouped per
    // interval like those of the Krylov blocks.
    // In the fixed-dimension mode the sweeps filter in the context's precision and keep
    // every Ritz vector; the refinement filters in FP64 and keeps the in-interval ones.
    int64_t refine_steps = 0;
    const int NBr = F > 1 ? NB : c->NBcap;  // columns of one refinement filter call
    const int gr = F > 1 ? g : NBr;         // of them per interval
    const bool sweep_fp64 = X0 ? c->opts.precision == KES_PREC_FP64 : true;
    auto keep = [&](const MeshSolve& m, int q) { return X0 != nullptr || !std::isnan(m.last_rel[q]); };
    for (int sweep = 0; sweep < so.refine_sweeps; ++sweep) {
      const bool from_x0 = X0 && sweep == 0;
      std::vector<int> pcount(P, 0);
      std::vector<int64_t> xoff(F + 1, 0);  // interval f uses columns xoff[f] .. of Xd (meshes share them)
      int rounds = 0;
      for (int p = 0; p < P; ++p) {
        if (from_x0) pcount[p] = p0;
        else
          for (size_t q = 0; q < ms[p].last_rel.size(); ++q) pcount[p] += keep(ms[p], static_cast<int>(q)) ? 1 : 0;
        rounds = std::max(rounds, (pcount[p] + gr - 1) / gr);
      }
      for (int f = 0; f < F; ++f) {
        int mx = 0;
        for (int j = 0; j < nm; ++j) mx = std::max(mx, pcount[j * F + f]);
        xoff[f + 1] = xoff[f] + mx;
      }
      if (xoff[F] == 0) break;
      const size_t need = static_cast<size_t>(xoff[F]) * np;
      if (need > c->Xd_cap) {
        c->dfree(c->Xd);
        c->Xd = c->dalloc_n<double>(need);
        c->Xd_cap = need;
      }
      KES_CUDA(cudaMemsetAsync(c->Xd, 0, need * sizeof(double), s));
      if (from_x0) {  // the caller's vectors, one column at a time into the padded row order
        for (int q = 0; q < p0; ++q) {
          const double* src = X0 + static_cast<int64_t>(q) * c->n;
          if (mem == KES_MEM_HOST) {
            KES_CUDA(cudaMemcpyAsync(c->tmp_user, src, static_cast<size_t>(c->n) * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
            src = c->tmp_user;
          }
          launch_gather_rows(s, src, c->n, 1, c->row_src, c->n, c->Xd + static_cast<int64_t>(q) * np, 1, np);
        }
        KES_CHECK_LAUNCH();
      }
      // Ritz vectors (all of them, or those of in-interval Ritz values): X = B y_q
      for (int p = 0; p < P && !from_x0; ++p) {
        if (pcount[p] == 0) continue;
        MeshSolve& m = ms[p];
        const MeshInfo& mi = mesh_of(p);
        const int kk = m.k;
        std::vector<double> theta, Y, Ysel;
        projected_eig(p, theta, Y);
        for (int q = 0; q < kk; ++q)
          if (keep(m, q))
            Ysel.insert(Ysel.end(), Y.begin() + static_cast<size_t>(q) * kk, Y.begin() + static_cast<size_t>(q + 1) * kk);
        KES_CUDA(cudaMemcpyAsync(c->Yd, Ysel.data(), Ysel.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        launch_gemm_bx(s, Bp(p), np, kk, c->Yd, pcount[p], c->Xd + xoff[p % F] * np + mi.row_off, np, mi.n_pad);
        KES_CHECK_LAUNCH();
        c->sync();  // Yd is reused by the next process
      }
      // filter them with the FP64 kernels, a block of NBr columns at a time, into fresh bases
      for (int p = 0; p < P; ++p) {
        want[p] = pcount[p] > 0;
        if (want[p]) {
          ms[p].k = 0;
          ms[p].done = false;
        }
      }
      std::vector<int32_t> csel(static_cast<size_t>(nm) * NBr, -1);
      for (int r = 0; r < rounds; ++r) {
        std::fill(csel.begin(), csel.end(), -1);
        for (int p = 0; p < P; ++p) {
          const int j = p / F, f = p % F;
          for (int i = 0; i < gr; ++i) {
            const int q = r * gr + i;
            if (q < pcount[p]) csel[j * NBr + f * gr + i] = static_cast<int32_t>(xoff[f] + q);
          }
        }
        KES_CUDA(cudaMemcpyAsync(c->colsel, csel.data(), csel.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        launch_pack_basis(s, c->Xd, np, c->colsel, c->slice_mesh, c->stage_in, NBr, np);
        KES_CHECK_LAUNCH();
        const int Lr = so.refine_L > 0 && so.refine_L < c->L ? so.refine_L : c->L;
        run_filter(c, NBr, sweep_fp64, cpt, Lr);
        refine_steps += Lr;
        launch_unpack_block(s, c->stage_out, NBr, c->Wc, np);
        KES_CHECK_LAUNCH();
        for (int jj = 0; jj < NBr; ++jj) {
          bool any = false;
          for (int j = 0; j < nm; ++j) {
            const int p = owner(j, jj);
            if (p < 0) continue;
            want[p] = csel[j * NBr + jj] >= 0;
            any |= want[p] != 0;
          }
          if (any) append_column(jj);
        }
      }
      std::vector<int> due;
      for (int p = 0; p < P; ++p) {
        if (pcount[p] > 0) due.push_back(p);
        want[p] = 1;
      }
      project_many(due);
    }

    // results: the pairs of a mesh's processes merged in ascending theta
    bool any_breakdown = false;
    for (int j = 0; j < nm; ++j) {
      const MeshInfo& mi = c->meshes[j];
      kes_result* r = res[j];
      struct Pair {
        double theta;
        int f, q;
      };
      std::vector<Pair> pairs;
      std::vector<double> ritz_th, ritz_rel;
      int k_used = 0;
      bool brk = false;
      for (int f = 0; f < F; ++f) {
        const MeshSolve& m = ms[j * F + f];
        for (size_t q = 0; q < m.acc_theta.size(); ++q) pairs.push_back({m.acc_theta[q], f, static_cast<int>(q)});
        ritz_th.insert(ritz_th.end(), m.last_theta.begin(), m.last_theta.end());
        ritz_rel.insert(ritz_rel.end(), m.last_rel.begin(), m.last_rel.end());
        k_used += m.k;
        brk |= m.breakdown;
      }
      std::stable_sort(pairs.begin(), pairs.end(), [](const Pair& x, const Pair& y) { return x.theta < y.theta; });
      const int np_acc = static_cast<int>(pairs.size());
      std::vector<double> th(np_acc), om(np_acc), rel(np_acc), ab(np_acc);
      std::vector<int32_t> iv(np_acc);
      for (int t = 0; t < np_acc; ++t) {
        const MeshSolve& m = ms[j * F + pairs[t].f];
        th[t] = pairs[t].theta;
        om[t] = std::sqrt(th[t]);
        rel[t] = m.acc_rel[pairs[t].q];
        ab[t] = m.acc_abs[pairs[t].q];
        iv[t] = pairs[t].f;
      }
      any_breakdown |= brk;
      r->n = mi.n;
      r->n_pairs = np_acc;
      r->k_used = k_used;
      r->breakdown = brk ? 1 : 0;
      r->n_ritz = static_cast<int32_t>(ritz_th.size());
      r->time_steps = steps;
      r->refine_steps = refine_steps;
      r->omega2 = hdup(th);
      r->omega = hdup(om);
      r->rel_res = hdup(rel);
      r->abs_res = hdup(ab);
      r->interval = hdup(iv);
      r->ritz_omega2 = hdup(ritz_th);
      r->ritz_rel_res = hdup(ritz_rel);
      if (so.want_vectors && np_acc > 0) {
        const size_t need = static_cast<size_t>(np_acc) * np;
        if (need > c->Xd_cap) {
          c->dfree(c->Xd);
          c->Xd = c->dalloc_n<double>(need);
          c->Xd_cap = need;
        }
        KES_CUDA(cudaMemsetAsync(c->Xd, 0, need * sizeof(double), s));
        // interval f's accepted vectors go to columns xo[f] .. of Xd
        std::vector<int> xo(F + 1, 0);
        for (int f = 0; f < F; ++f) {
          const MeshSolve& m = ms[j * F + f];
          const int cnt = static_cast<int>(m.acc_theta.size());
          xo[f + 1] = xo[f] + cnt;
          if (cnt == 0) continue;
          KES_CUDA(cudaMemcpyAsync(c->Yd, m.acc_Y.data(), m.acc_Y.size() * sizeof(double), cudaMemcpyHostToDevice, s));
          launch_gemm_bx(s, Bp(j * F + f), np, m.k, c->Yd, cnt, c->Xd + static_cast<int64_t>(xo[f]) * np + mi.row_off,
                         np, mi.n_pad);
          KES_CHECK_LAUNCH();
          c->sync();  // Yd is reused by the next interval
        }
        r->vectors = static_cast<double*>(std::malloc(static_cast<size_t>(np_acc) * mi.n * sizeof(double)));
        if (!r->vectors) throw std::bad_alloc();
        // scatter each Ritz vector to the caller's order and keep this mesh's rows
        for (int t = 0; t < np_acc; ++t) {
          const int64_t col = xo[pairs[t].f] + pairs[t].q;
          launch_scatter_rows(s, c->Xd + col * np, 1, 1, c->row_src, c->n, c->tmp_user, c->n, np);
          KES_CHECK_LAUNCH();
          KES_CUDA(cudaMemcpyAsync(r->vectors + static_cast<size_t>(t) * mi.n, c->tmp_user + mi.src_off,
                                   mi.n * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        c->sync();
      }
    }
    c->sync();
    return any_breakdown ? KES_INFO_INVARIANT_SUBSPACE : KES_OK;
  });
  const double ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (st != KES_OK && st != KES_INFO_INVARIANT_SUBSPACE) {
    for (auto* r : res) kes_result_free(r);
    return st;
  }
  for (int j = 0; j < nm; ++j) {
    res[j]->solve_ms = ms_total;
    out[j] = res[j];
  }
  return st;
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
  o->compact_cols = 1;
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
  return create_impl(out, 1, &n, &row_ptr, &col, &val, &m_diag, opts);
}

kes_status kes_create_batch(kes_ctx** out, int32_t n_mesh, const int64_t* n, const int64_t* const* row_ptr,
                            const int32_t* const* col, const double* const* val, const double* const* m_diag,
                            const kes_opts* opts) {
  return create_impl(out, n_mesh, n, row_ptr, col, val, m_diag, opts);
}

void kes_destroy(kes_ctx* ctx) { release(ctx); }

int64_t kes_size(const kes_ctx* ctx) { return ctx ? ctx->n : -1; }

int32_t kes_mesh_count(const kes_ctx* ctx) { return ctx ? ctx->n_mesh() : -1; }

kes_status kes_sync(kes_ctx* ctx) {
  if (!ctx) return KES_ERR_ARG;
  return guarded([&]() -> kes_status { return check_flag(ctx); });
}

void kes_launch_shapes(int32_t* n_step, int32_t* n_block) {
  if (n_step) *n_step = step_variant_count();
  if (n_block) *n_block = blk_variant_count();
}

int64_t kes_step_bytes(const kes_ctx* c, int32_t b, int32_t F) {
  if (!c || b < 1 || F < 1) return -1;
  // matrix: value (of A = -tau^2 M^{-1} S) + int32 column per stored entry, plus a 4-byte
  // row pointer per row as CSR would need; per row and vector: the gather of u_n once,
  // u_{n-1} read, u_{n+1} written, F accumulators read and written (FP32 form: s and c).
  // The fourth-order stepper adds a stage pass (matrix and row pointers again, u_n gathered,
  // the stage written) and the step reads the stage (gathered) besides u_n. With the
  // compact index a stored entry's column takes 2 bytes instead of 4.
  const int64_t vs = c->opts.precision == KES_PREC_FP64 ? 8 : 4;
  const int64_t is = c->A.dcol ? 2 : 4;
  const int64_t mat = (vs + is) * c->nnz + 4 * (c->n + 1);
  const int64_t step = mat + c->n * int64_t(b) * (3 * vs + 16 * F);
  if (c->opts.stepper == KES_STEPPER_LEAPFROG4) return step + mat + c->n * int64_t(b) * (3 * vs);
  return step;
}

kes_status kes_estimate_omega_max(kes_ctx* c, int32_t iters, const double* v0, double* omega_max,
                                  double* gershgorin) {
  if (!c || !v0 || !omega_max || iters < 0) return KES_ERR_ARG;
  if (c->n_mesh() != 1) return KES_ERR_UNSUPPORTED;
  return omega_impl(c, iters, v0, omega_max, gershgorin);
}

kes_status kes_estimate_omega_max_batch(kes_ctx* c, int32_t iters, const double* v0, double* omega_max,
                                        double* gershgorin) {
  if (!c || !v0 || !omega_max || iters < 0) return KES_ERR_ARG;
  return omega_impl(c, iters, v0, omega_max, gershgorin);
}

kes_status kes_set_filters(kes_ctx* c, int32_t F, const double* wmin, const double* wmax, double tau, int32_t L) {
  if (!c || F < 1 || !wmin || !wmax || L < 1) return KES_ERR_ARG;
  const int nm = c->n_mesh();
  std::vector<double> a(static_cast<size_t>(nm) * F), b(a.size()), t(nm, tau);
  for (int j = 0; j < nm; ++j)
    for (int f = 0; f < F; ++f) {
      a[j * F + f] = wmin[f];
      b[j * F + f] = wmax[f];
    }
  return set_weights_impl(c, F, nullptr, a.data(), b.data(), t.data(), L);
}

kes_status kes_set_filter(kes_ctx* c, double wmin, double wmax, double tau, int32_t L) {
  return kes_set_filters(c, 1, &wmin, &wmax, tau, L);
}

kes_status kes_set_filters_batch(kes_ctx* c, int32_t F, const double* wmin, const double* wmax, const double* tau,
                                 int32_t L) {
  if (!c || F < 1 || !wmin || !wmax || !tau || L < 1) return KES_ERR_ARG;
  return set_weights_impl(c, F, nullptr, wmin, wmax, tau, L);
}

kes_status kes_set_weights(kes_ctx* c, int32_t F, const double* alpha, const double* wmin, const double* wmax,
                           const double* tau, int32_t L) {
  if (!c || F < 1 || !alpha || !wmin || !wmax || !tau || L < 1) return KES_ERR_ARG;
  return set_weights_impl(c, F, alpha, wmin, wmax, tau, L);
}

kes_status kes_alpha_gaussian(double center, double sigma, double tau, int32_t L, double* alpha) {
  if (!alpha || L < 1 || !(tau > 0.0) || !(sigma > 0.0) || !(center >= 0.0) || !std::isfinite(center))
    return KES_ERR_ARG;
  kes::alpha_gaussian(center, sigma, tau, L, alpha);
  return KES_OK;
}

kes_status kes_alpha_triangle(double center, double half_width, double tau, int32_t L, double* alpha) {
  if (!alpha || L < 1 || !(tau > 0.0) || !(half_width > 0.0) || !(center >= 0.0) || !std::isfinite(center) ||
      !std::isfinite(half_width))
    return KES_ERR_ARG;
  kes::alpha_triangle(center, half_width, tau, L, alpha);
  return KES_OK;
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

kes_status kes_weights_response(const double* alpha, double tau, int32_t L, const double* omega, int64_t k,
                                double* beta) {
  if (!alpha || !omega || !beta || k < 0 || L < 1 || !(tau > 0.0)) return KES_ERR_ARG;
  kes::weights_response(alpha, tau, L, omega, k, beta);
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
  LaunchCount lc(&c->stats);
  return guarded([&]() -> kes_status {
    const int NB = nb_for(b);
    block_in(c, r_in, b, mem, NB, c->stage_in);
    run_filter(c, NB, c->opts.precision == KES_PREC_FP64);
    for (int f = 0; f < c->F; ++f)
      block_out(c, c->stage_out + static_cast<int64_t>(f) * c->n_pad * NB, NB, b,
                r_out + static_cast<int64_t>(f) * b * c->n, mem);
    KES_CHECK_LAUNCH();
    if (mem == KES_MEM_HOST) return check_flag(c);
    return KES_OK;
  });
}

kes_status kes_filter_apply_columns(kes_ctx* c, const double* r_in, double* r_out, int32_t b, int32_t mem) {
  if (!c || !r_in || !r_out || b < 2 || b > c->opts.block_b || (mem != KES_MEM_HOST && mem != KES_MEM_DEVICE))
    return KES_ERR_ARG;
  if (!c->filter_set) return KES_ERR_STATE;
  if (b % c->F != 0) return KES_ERR_ARG;
  LaunchCount lc(&c->stats);
  return guarded([&]() -> kes_status {
    const int NB = nb_for(b);
    block_in(c, r_in, b, mem, NB, c->stage_in);
    run_filter(c, NB, c->opts.precision == KES_PREC_FP64, b / c->F);
    block_out(c, c->stage_out, NB, b, r_out, mem);
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
  std::free(r->interval);
  std::free(r);
}

kes_status kes_krylov_solve(kes_ctx* c, const double* r0, int32_t mem, const kes_solve_opts* so_in,
                            kes_result** out) {
  if (!c || !r0 || !out || (mem != KES_MEM_HOST && mem != KES_MEM_DEVICE)) return KES_ERR_ARG;
  *out = nullptr;
  if (!c->filter_set) return KES_ERR_STATE;
  if (c->F != 1 || c->n_mesh() != 1) return KES_ERR_UNSUPPORTED;
  kes_solve_opts so;
  if (so_in) so = *so_in;
  else kes_solve_opts_default(&so);
  if (so.kmax < 1 || so.check_every < 1 || !(so.tol > 0.0) || so.refine_sweeps < 0 || so.refine_L < 0)
    return KES_ERR_ARG;
  return block_solve_impl(c, r0, 1, mem, so, out);
}

kes_status kes_block_krylov_solve(kes_ctx* c, const double* R0, int32_t b, int32_t mem, const kes_solve_opts* so_in,
                                  kes_result** out) {
  if (!c || !R0 || !out || b < 1 || b > c->opts.block_b || (mem != KES_MEM_HOST && mem != KES_MEM_DEVICE))
    return KES_ERR_ARG;
  for (int j = 0; j < c->n_mesh(); ++j) out[j] = nullptr;
  if (!c->filter_set) return KES_ERR_STATE;
  if (b % c->F != 0) return KES_ERR_ARG;
  kes_solve_opts so;
  if (so_in) so = *so_in;
  else kes_solve_opts_default(&so);
  if (so.kmax < b / c->F || so.check_every < 1 || !(so.tol > 0.0) || so.refine_sweeps < 0 || so.refine_L < 0)
    return KES_ERR_ARG;
  return block_solve_impl(c, R0, b, mem, so, out);
}

kes_status kes_subspace_solve(kes_ctx* c, const double* X0, int32_t p, int32_t mem, const kes_solve_opts* so_in,
                              kes_result** out) {
  if (!c || !X0 || !out || p < 1 || (mem != KES_MEM_HOST && mem != KES_MEM_DEVICE)) return KES_ERR_ARG;
  for (int j = 0; j < c->n_mesh(); ++j) out[j] = nullptr;
  if (!c->filter_set) return KES_ERR_STATE;
  if (c->F != 1) return KES_ERR_UNSUPPORTED;
  kes_solve_opts so;
  if (so_in) so = *so_in;
  else kes_solve_opts_default(&so);
  if (so.kmax < p || so.refine_sweeps < 1 || !(so.tol > 0.0) || so.refine_L < 0) return KES_ERR_ARG;
  return block_solve_impl(c, nullptr, 1, mem, so, out, X0, p);
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
    c->stats.blk_variant = c->NBcap > 1 ? c->cfg.variant_blk : -1;
    c->stats.blk_grid = c->NBcap > 1 ? c->cfg.grid_blk : 0;
    return KES_OK;
  });
}

}  // extern "C"
