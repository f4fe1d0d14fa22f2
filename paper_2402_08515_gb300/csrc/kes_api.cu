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

#include "kes_ctx.h"

using namespace kes;

namespace {

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
}  // namespace

namespace kes {

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

}  // namespace kes

namespace {

// --------------------------------------------------------------- filter
// Largest stable tau * omega of the context's stepper.
double cfl_bound(const kes_ctx* c) { return c->opts.stepper == KES_STEPPER_LEAPFROG4 ? 2.0 * std::sqrt(3.0) : 2.0; }

// Issues the fused steps of one filter application of an NB-column block on the context
// stream: stage_in -> stage_out (cpt = 0: F filtered blocks, every column with every
// weight table; cpt > 0: one block, column j with table min(j / cpt, F - 1)). steps <= L
// runs the first steps + 1 weights of the tables: alpha(t) of eq. (weightf) does not
// depend on T, so that is the filter of end time steps * tau.
int64_t issue_filter_steps(kes_ctx* c, int NB, bool fp64, int cpt, int steps, bool x2) {
  const int64_t before = g_launches;
  const bool ho = c->opts.stepper == KES_STEPPER_LEAPFROG4;
  const int L = c->L, F = c->F;  // L: the tables' length (their stride is L + 1)
  const int64_t stride = c->n_pad * NB;
  if (x2) {
    // FP32 pairs: the FP64 step values (fold64 as for the FP64 steps) split once per filter
    const SellDev A64 = c->step_A64();
    launch_init_x2(c->stream, c->A, NB, c->stage_in, c->U2[2], c->acc_s, c->acc_c, stride, F, c->alpha64, L, cpt);
    int next = 1;  // the initialisation added alpha_0 u_0
    for (int s = 0; s < steps; ++s) {
      const bool first = s == 0, last = s == steps - 1;
      const float2* x = s == 0 ? c->U2[2] : c->U2[(s - 1) & 1];
      const float2* prev = s <= 1 ? c->U2[2] : c->U2[s & 1];
      float2* out = c->U2[s & 1];
      bool init = false;
      const int nterm = acc_plan(s, steps, next, init);
      launch_step_x2(A64, c->cfg, c->stream, NB, first, last, c->step2, x, prev, out, c->acc_s, c->acc_c,
                     c->stage_out, stride, F, c->alpha_hi, c->alpha_lo, L, s, cpt, nterm, c->d_flag);
    }
  } else if (fp64) {
    // in a context of the FP32 form the launch shape was tuned for the FP32 kernels:
    // the FP64 steps of the refinement take a fixed register-staged shape
    const SellDev A64 = c->step_A64();
    LaunchCfg cfg = c->cfg;
    if (c->opts.precision != KES_PREC_FP64) {
      cfg.variant = 3;
      cfg.grid_step = cfg.n_sm * step_blocks_per_sm(false, 3, cfg.block_step);
    }
    int next = 0;  // first weighted term not yet in the accumulators
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
      bool init = false;
      const int nterm = acc_plan(s, steps, next, init);
      if (NB == 1) {
        launch_step_f64(A64, cfg, c->stream, first, x, g, prev, out, c->stage_out, stride, F, c->alpha64, L, s,
                        last, nterm, init, c->d_flag);
      } else {
        launch_step_blk_f64(A64, cfg, c->stream, NB, first, last, x, g, prev, out, c->stage_out, stride, F,
                            c->alpha64, L, s, cpt, nterm, init, c->d_flag);
      }
    }
  } else {
    const SellDev A32 = c->step_A32();
    launch_init_f32(c->stream, c->A, NB, c->stage_in, c->U32[2], c->acc_s, c->acc_c, stride, F, c->alpha64, L, cpt);
    int next = 1;  // the initialisation added alpha_0 u_0
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
      bool init = false;
      const int nterm = acc_plan(s, steps, next, init);
      if (NB == 1) {
        launch_step_f32(A32, c->cfg, c->stream, first, last, x, g, prev, out, c->acc_s, c->acc_c, c->stage_out,
                        stride, F, c->alpha_hi, c->alpha_lo, L, s, nterm, c->d_flag);
      } else {
        launch_step_blk_f32(A32, c->cfg, c->stream, NB, first, last, x, g, prev, out, c->acc_s, c->acc_c,
                            c->stage_out, stride, F, c->alpha_hi, c->alpha_lo, L, s, cpt, nterm, c->d_flag);
      }
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

// The FP32-pair steps in a context of the FP32 form: step values split from the FP64 ones
// (again after a filter change rescaled those) and the pair state.
void ensure_x2_state(kes_ctx* c) {
  ensure_fp64_state(c);
  if (!c->step2) c->step2 = c->dzero_n<float2>(c->nnz_pad);
  if (!c->step2_fresh) {
    launch_split_values(c->stream, c->nnz_pad, c->step64, c->step2);
    KES_CHECK_LAUNCH();
    c->step2_fresh = true;
  }
  if (!c->U2[0])
    for (int j = 0; j < 3; ++j) c->U2[j] = c->dzero_n<float2>(c->n_pad * c->NBcap);
}

}  // namespace

namespace kes {

void run_filter(kes_ctx* c, int NB, bool fp64, int cpt, int steps, bool x2) {
  if (cpt > 0 && NB < 2) throw KesError{KES_ERR_ARG};  // per-column tables live in the block kernels
  if (x2 && (NB < 2 || c->opts.precision != KES_PREC_FP32 || c->opts.stepper != KES_STEPPER_LEAPFROG))
    throw KesError{KES_ERR_UNSUPPORTED};
  if (steps <= 0 || steps > c->L) steps = c->L;
  if (x2) ensure_x2_state(c);
  else if (fp64) ensure_fp64_state(c);
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
      if (g.NB == NB && g.fp64 == fp64 && g.x2 == x2 && g.cpt == cpt && g.steps == steps) ge = &g;
    if (!ge) {
      cudaGraph_t graph;
      KES_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      const int64_t nodes = issue_filter_steps(c, NB, fp64, cpt, steps, x2);
      cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
      g_launches -= nodes;  // captured, not launched
      KES_CUDA(ce);
      GraphEntry g;
      g.NB = NB;
      g.fp64 = fp64;
      g.x2 = x2;
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
    issue_filter_steps(c, NB, fp64, cpt, steps, x2);
    KES_CHECK_LAUNCH();
  }
  KES_CUDA(cudaEventRecord(e1, c->stream));
  c->ev_filter.emplace_back(e0, e1);
  c->stats.filter_calls += 1;
  c->stats.filter_steps += steps;
}

}  // namespace kes

namespace {

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
}  // namespace

namespace kes {

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
  // partial sums: every process's inner products of one batched stage at once (a process
  // takes dot_blocks of its rows per column), and the single launches' kDotBlocks per column
  int64_t dot_total = 0;
  for (const MeshInfo& mi : c->meshes) dot_total += static_cast<int64_t>(F) * dot_blocks(mi.n_pad);
  c->partial = c->dalloc_n<double>(std::max(nproc * kDotBlocks, dot_total) * (2 * kmax + 8));
  c->normd = c->dzero_n<double>(2 * nproc);
  // job descriptors of the batched Gram-Schmidt stages (see append_column)
  c->jobs_bytes = static_cast<size_t>(nproc) * (4 * sizeof(DotJob) + sizeof(GemvJob) + sizeof(ScaleJob)) +
                  static_cast<size_t>(2 * F * c->n_mesh()) * sizeof(double*) + 256;
  c->jobs = static_cast<char*>(c->dalloc(c->jobs_bytes));
  c->scal = c->dzero_n<double>(nproc * (2 * kmax + kScal));
  c->Yd = c->dalloc_n<double>(nproc * kmax * kmax);  // every process's selected Ritz vectors at once
  c->thd = c->dalloc_n<double>(nproc * kmax);
}

}  // namespace kes

namespace {


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
  // single-vector kernel, over the middle steps of a filter application: two that leave
  // the accumulators alone, one that adds three terms
  int best = 0;
  float best_ms = 3.0e38f;
  for (int v = 0; v < step_variant_count(); ++v) {
    select_variant(c, v);
    const float ms = timed([&](int count) {
      for (int i = 0; i < count; ++i) {
        const int nterm = i % 3 == 2 ? 3 : 0;
        if (fp32)
          launch_step_f32(c->step_A32(), c->cfg, c->stream, false, false, c->U32[0], c->U32[0], c->U32[1], c->U32[1],
                          c->acc_s, c->acc_c, c->stage_out, c->n_pad, 1, a32, a32, 7, 1, nterm, c->d_flag);
        else
          launch_step_f64(c->step_A64(), c->cfg, c->stream, false, c->U64[0], c->U64[0], c->U64[1], c->U64[1],
                          c->stage_out, c->n_pad, 1, a64, 7, 1, false, nterm, false, c->d_flag);
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
          // the middle steps of a filter application: two that leave the accumulators
          // alone, one that adds three terms
          const int nterm = i % 3 == 2 ? 3 : 0;
          if (fp32)
            launch_step_blk_f32(c->step_A32(), c->cfg, c->stream, NB, false, false, c->U32[0], c->U32[0], c->U32[1],
                                c->U32[1], c->acc_s, c->acc_c, c->stage_out, c->n_pad * NB, 1, a32, a32, 7, 1, 0,
                                nterm, c->d_flag);
          else
            launch_step_blk_f64(c->step_A64(), c->cfg, c->stream, NB, false, false, c->U64[0], c->U64[0], c->U64[1],
                                c->U64[1], c->stage_out, c->n_pad * NB, 1, a64, 7, 1, 0, nterm, false, c->d_flag);
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
    c->step2_fresh = false;  // the FP32-pair values follow step64 at their next use
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
  // The step kernels read and write the accumulators only in the steps that add the weighted
  // terms (every third step and the last, acc_plan): their 16 F bytes count with that share of
  // a filter application of the context's L steps.
  const int64_t vs = c->opts.precision == KES_PREC_FP64 ? 8 : 4;
  const int64_t is = c->A.dcol ? 2 : 4;
  const int64_t mat = (vs + is) * c->nnz + 4 * (c->n + 1);
  int64_t acc = c->n * int64_t(b) * 16 * F;
  if (c->L > 0) {
    int next = vs == 8 ? 0 : 1, n_acc = 0;
    bool init = false;
    for (int s = 0; s < c->L; ++s) n_acc += acc_plan(s, c->L, next, init) > 0;
    acc = acc * n_acc / c->L;
  }
  const int64_t step = mat + c->n * int64_t(b) * 3 * vs + acc;
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

// Refinement sweeps in FP32 pairs need a context of the FP32 form with block columns (the
// sweep's filter is a block kernel) and the leapfrog stepper; checked before the Krylov phase.
static bool refine_precision_supported(const kes_ctx* c, const kes_solve_opts& so) {
  if (so.refine_precision != KES_REFINE_F32X2 || so.refine_sweeps == 0 || c->opts.precision != KES_PREC_FP32)
    return true;
  return c->opts.stepper == KES_STEPPER_LEAPFROG && (c->F > 1 || c->NBcap >= 2);
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
  if (so.kmax < 1 || so.check_every < 1 || !(so.tol > 0.0) || so.refine_sweeps < 0 || so.refine_L < 0 ||
      so.refine_extra < 0 ||
      (so.refine_precision != KES_REFINE_FP64 && so.refine_precision != KES_REFINE_F32X2))
    return KES_ERR_ARG;
  if (so.kmax > kMaxProjected || !refine_precision_supported(c, so)) return KES_ERR_UNSUPPORTED;
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
  if (so.kmax < b / c->F || so.check_every < 1 || !(so.tol > 0.0) || so.refine_sweeps < 0 || so.refine_L < 0 ||
      so.refine_extra < 0 ||
      (so.refine_precision != KES_REFINE_FP64 && so.refine_precision != KES_REFINE_F32X2))
    return KES_ERR_ARG;
  if (so.kmax > kMaxProjected || !refine_precision_supported(c, so)) return KES_ERR_UNSUPPORTED;
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
  if (so.kmax < p || so.refine_sweeps < 1 || !(so.tol > 0.0) || so.refine_L < 0 || so.refine_extra < 0 ||
      (so.refine_precision != KES_REFINE_FP64 && so.refine_precision != KES_REFINE_F32X2))
    return KES_ERR_ARG;
  if (so.kmax > kMaxProjected || !refine_precision_supported(c, so)) return KES_ERR_UNSUPPORTED;
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
