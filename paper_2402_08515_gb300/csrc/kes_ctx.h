// The context of the kes library (struct kes_ctx) and the helpers that the context
// code (kes_api.cu) and the eigensolver (solver.cu) share. Internal: not part of the
// C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <exception>
#include <new>
#include <utility>
#include <vector>

#include "kes_internal.h"

namespace kes {

struct KesError {
  kes_status status;
};

#define KES_CUDA(call)                                                \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) {                                          \
      throw ::kes::KesError{e_ == cudaErrorMemoryAllocation ? KES_ERR_OOM \
                                                            : KES_ERR_CUDA}; \
    }                                                                 \
  } while (0)

#define KES_CHECK_LAUNCH() KES_CUDA(cudaGetLastError())

template <typename F>
inline kes_status guarded(F&& f) {
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
  bool x2 = false;
  int cpt = 0;
  int steps = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t nodes = 0;
};

inline int nb_for(int b) { return b <= 1 ? 1 : b <= 2 ? 2 : b <= 4 ? 4 : 8; }

}  // namespace kes

struct kes_ctx {
  kes_opts opts{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  std::vector<kes::MeshInfo> meshes;
  int64_t n = 0, n_pad = 0, nnz = 0, nnz_pad = 0;
  std::vector<std::pair<void*, size_t>> allocs;
  kes::SellDev A;
  kes::LaunchCfg cfg;
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
  kes::SellDev step_A64() const {
    kes::SellDev a = A;
    a.val64 = step64;
    a.val64p = step64p;
    a.fold2 = fold64 ? 1 : 0;
    return a;
  }
  kes::SellDev step_A32() const {
    kes::SellDev a = A;
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
  // FP32-pair refinement filter (allocated on first use): step values split from step64,
  // state ping-pong [0], [1] and start [2] (n_pad x NBcap pairs each)
  float2* step2 = nullptr;
  bool step2_fresh = false;  // step2 holds the current step64
  float2* U2[3] = {nullptr, nullptr, nullptr};
  float* V32 = nullptr;
  float* acc_s = nullptr;
  float* acc_c = nullptr;
  double* tmp_user = nullptr;  // n x NBcap, caller layout
  int* d_flag = nullptr;
  std::vector<kes::GraphEntry> graphs;
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
      if (!p) throw kes::KesError{KES_ERR_OOM};
    } else {
      cudaError_t e = cudaMalloc(&p, bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        throw kes::KesError{KES_ERR_OOM};
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


namespace kes {

constexpr int kScal = 16;  // device scalars per process ahead of the Gram-Schmidt coefficients

// Caller block (n x nb column-major, host or device) -> row-major n_pad x NB block.
void block_in(kes_ctx* c, const double* src, int nb, int32_t mem, int NB, double* dst);
// Row-major n_pad x NB block (first nb columns) -> caller block (n x nb column-major).
void block_out(kes_ctx* c, const double* src, int NB, int nb, double* dst, int32_t mem);
// One filter application of an NB-column block on the context stream: stage_in ->
// stage_out (cpt = 0: F filtered blocks; cpt > 0: column j with weight table j / cpt),
// the first `steps` steps of the installed tables (0: all L), as a CUDA graph if enabled.
// x2: in FP32 pairs (FP32-form contexts, NB >= 2, leapfrog; fp64 is then ignored).
void run_filter(kes_ctx* c, int NB, bool fp64, int cpt = 0, int steps = 0, bool x2 = false);
// Krylov workspace for kmax basis vectors per process and F intervals per mesh.
void ensure_krylov(kes_ctx* c, int kmax, int F);
// Device scalars of process p (of mesh p outside the solver).
inline double* proc_scal(kes_ctx* c, int p) { return c->scal + static_cast<int64_t>(p) * (2 * c->kcap + kScal); }

// The block Krylov eigensolver (Algorithm 2.5 and its block version in Sec. 4) over every
// mesh and interval of the context, and its fixed-dimension mode (X0); see solver.cu.
kes_status block_solve_impl(kes_ctx* c, const double* R0, int b, int32_t mem, const kes_solve_opts& so,
                            kes_result** out, const double* X0 = nullptr, int p0 = 0);

}  // namespace kes
