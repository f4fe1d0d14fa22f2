// The block Krylov eigensolver of the kes library (Nannen & Wess, arXiv:2402.08515):
// Algorithm 2.5 (Krylov space by filtered time-domain solutions) and its block version
// of Sec. 4, for every mesh and interval of a context, with the fixed-dimension
// (FEAST-like) use of the filter of Sec. 4 as refinement or as a solver of its own.
//
// The solve runs in stages, one method each:
//   start      the start block, M-orthonormalised (the first basis vectors)
//   krylov     block steps: filter the newest basis vectors (run_filter), orthogonalise
//              the filtered block into the basis (orthogonalise), project when due
//   project    Rayleigh-Ritz (eq. projevp) and the residual acceptance (eq. res)
//   refine     sweeps of filtered subspace iteration on Ritz vectors
//   results    the accepted pairs of each mesh, merged over its intervals
//
// Process p = mesh * F + f is the block Krylov iteration of mesh p / F on interval f from
// start columns f * g .. f * g + g - 1 (g = b / F), with its own basis, Gram-Schmidt
// scalars and projected matrix; the processes share only the b-column trajectory of each
// block step.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

#include "kes_ctx.h"

namespace kes {
namespace {

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

class BlockSolver {
 public:
  // X0 (p0 caller vectors, n_total x p0 column-major) selects the fixed-dimension mode.
  BlockSolver(kes_ctx* c, int b, const kes_solve_opts& so, const double* X0, int p0)
      : c_(c), so_(so), X0_(X0), p0_(p0), nm_(c->n_mesh()), F_(c->F), P_(nm_ * F_), b_(b), g_(b / F_),
        cpt_(F_ > 1 ? g_ : 0), kmax_(so.kmax), NB_(nb_for(b)), ms_(P_), want_(P_, 1), np_(c->n_pad),
        kc_(c->kcap), s_(c->stream) {}

  void start(const double* R0, int32_t mem);
  void krylov();
  void refine(int32_t mem);
  bool results(std::vector<kes_result*>& res);

 private:
  std::vector<char> orthogonalise(int jj);
  void projected_eig(int p, std::vector<double>& theta, std::vector<double>& Y);
  void project(const std::vector<int>& ps);
  void check_wanted();

  cudaEvent_t other_begin() {
    cudaEvent_t e0 = c_->get_event();
    KES_CUDA(cudaEventRecord(e0, s_));
    return e0;
  }
  void other_end(cudaEvent_t e0) {
    cudaEvent_t e1 = c_->get_event();
    KES_CUDA(cudaEventRecord(e1, s_));
    c_->ev_other.emplace_back(e0, e1);
  }
  const MeshInfo& mesh_of(int p) const { return c_->meshes[p / F_]; }
  // column 0 of process p's basis over all rows (SpMV input) and on its mesh's rows
  double* Bfull(int p) const { return c_->B + (p % F_) * kc_ * np_; }
  double* Bp(int p) const { return Bfull(p) + mesh_of(p).row_off; }
  double* SBp(int p) const { return c_->SB + (p % F_) * kc_ * np_ + mesh_of(p).row_off; }
  double* Hcol(int p, int k) const { return c_->Hd + (static_cast<int64_t>(p) * kc_ + k) * kc_; }
  // process that owns column jj of a block of mesh j (-1: a padding column)
  int owner(int j, int jj) const {
    const int f = F_ > 1 ? jj / g_ : 0;
    return f < F_ ? j * F_ + f : -1;
  }

  kes_ctx* c_;
  const kes_solve_opts& so_;
  const double* X0_;
  const int p0_;
  const int nm_, F_, P_, b_, g_, cpt_, kmax_, NB_;
  std::vector<MeshSolve> ms_;
  std::vector<char> want_;  // processes taking part in the current block step
  const int64_t np_, kc_;
  cudaStream_t s_;
  int64_t steps_ = 0, refine_steps_ = 0;
};

// Orthogonalises column jj of Wc against the basis of the process that owns it on each
// mesh (two classical passes in the M-inner product) and appends the vectors that are
// not dependent (Algorithm 2.5). Returns the processes that gained a vector.
std::vector<char> BlockSolver::orthogonalise(int jj) {
  std::vector<char> added(P_, 0);
  std::vector<int> act;  // processes that take column jj
  for (int j = 0; j < nm_; ++j) {
    const int p = owner(j, jj);
    if (p < 0 || !want_[p] || ms_[p].done || ms_[p].k >= kmax_) continue;
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
    double* w = c_->Wc + static_cast<int64_t>(jj) * np_ + mi.row_off;
    const double* mj = c_->m64 + mi.row_off;
    const int nblk = dot_blocks(mi.n_pad), gblk = gemv_blocks(mi.n_pad);
    nb_jobs[i] = DotJob{w, w, mj, c_->normd + 2 * p, mi.n_pad, 0, poff, 0, 1, nblk};
    na_jobs[i] = DotJob{w, w, mj, c_->normd + 2 * p + 1, mi.n_pad, 0, poff, 0, 1, nblk};
    poff += nblk;
    const int k = ms_[p].k;
    if (k > 0) {
      h_jobs.push_back(DotJob{Bp(p), w, mj, proc_scal(c_, p) + kScal, mi.n_pad, np_, poff_h, 0, k, nblk});
      g_jobs.push_back(GemvJob{w, Bp(p), proc_scal(c_, p) + kScal, mi.n_pad, np_, 0, k, gblk});
      poff_h += static_cast<int64_t>(k) * nblk;
      max_k = std::max(max_k, k);
    }
  }
  const int nh = static_cast<int>(h_jobs.size());
  const int64_t nb_blocks = first_blocks(nb_jobs), na_blocks = first_blocks(na_jobs);
  const int64_t h_blocks = first_blocks(h_jobs), g_blocks = first_blocks(g_jobs);
  char* jb = c_->jobs;
  DotJob* d_nb = reinterpret_cast<DotJob*>(jb);
  DotJob* d_na = d_nb + P_;
  DotJob* d_h = d_na + P_;
  GemvJob* d_g = reinterpret_cast<GemvJob*>(d_h + P_);
  cudaEvent_t ev = other_begin();
  KES_CUDA(cudaMemcpyAsync(d_nb, nb_jobs.data(), na * sizeof(DotJob), cudaMemcpyHostToDevice, s_));
  KES_CUDA(cudaMemcpyAsync(d_na, na_jobs.data(), na * sizeof(DotJob), cudaMemcpyHostToDevice, s_));
  if (nh > 0) {
    KES_CUDA(cudaMemcpyAsync(d_h, h_jobs.data(), nh * sizeof(DotJob), cudaMemcpyHostToDevice, s_));
    KES_CUDA(cudaMemcpyAsync(d_g, g_jobs.data(), nh * sizeof(GemvJob), cudaMemcpyHostToDevice, s_));
  }
  launch_mdot_jobs(s_, d_nb, na, 1, nb_blocks, c_->partial);  // ||w||_M^2 before
  for (int pass = 0; pass < 2 && nh > 0; ++pass) {
    launch_mdot_jobs(s_, d_h, nh, max_k, h_blocks, c_->partial);  // h = B^T M w
    launch_gemv_sub_jobs(s_, d_g, nh, max_k, g_blocks);           // w -= B h
  }
  launch_mdot_jobs(s_, d_na, na, 1, na_blocks, c_->partial);  // ||w||_M^2 after
  KES_CHECK_LAUNCH();
  std::vector<double> nrm(2 * P_, 0.0);
  KES_CUDA(cudaMemcpyAsync(nrm.data(), c_->normd, 2 * P_ * sizeof(double), cudaMemcpyDeviceToHost, s_));
  int flag = 0;
  KES_CUDA(cudaMemcpyAsync(&flag, c_->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s_));
  other_end(ev);
  c_->sync();
  if (flag) {
    KES_CUDA(cudaMemsetAsync(c_->d_flag, 0, sizeof(int), s_));
    throw KesError{KES_ERR_UNSTABLE};
  }
  // phase 2 for the vectors that are not dependent: b_k = w / ||w||_M, S b_k (one
  // launch per interval over all meshes), the new column b_i^T S b_k of H
  std::vector<ScaleJob> s_jobs;
  std::vector<DotJob> c_jobs;
  std::vector<const double*> x_of(static_cast<size_t>(F_) * nm_, nullptr);
  std::vector<double*> y_of(static_cast<size_t>(F_) * nm_, nullptr);
  int max_k1 = 0, max_sblk = 1;
  poff = 0;
  for (int i = 0; i < na; ++i) {
    const int p = act[i];
    if (!(std::sqrt(nrm[2 * p + 1]) > 1e-10 * std::sqrt(nrm[2 * p]))) continue;  // dependent vector
    const MeshInfo& mi = mesh_of(p);
    const int k = ms_[p].k;
    double* w = c_->Wc + static_cast<int64_t>(jj) * np_ + mi.row_off;
    double* sbk = SBp(p) + k * np_;
    const int nblk = dot_blocks(mi.n_pad);
    s_jobs.push_back(ScaleJob{w, c_->normd + 2 * p + 1, Bp(p) + k * np_, mi.n_pad});
    max_sblk = std::max(max_sblk, gemv_blocks(mi.n_pad));
    x_of[static_cast<size_t>(p % F_) * nm_ + p / F_] = Bfull(p) + k * np_;
    y_of[static_cast<size_t>(p % F_) * nm_ + p / F_] = c_->SB + (p % F_) * kc_ * np_ + k * np_;
    c_jobs.push_back(DotJob{Bp(p), sbk, nullptr, Hcol(p, k), mi.n_pad, np_, poff, 0, k + 1, nblk});
    poff += static_cast<int64_t>(k + 1) * nblk;
    max_k1 = std::max(max_k1, k + 1);
    ms_[p].k = k + 1;
    added[p] = 1;
  }
  const int ns = static_cast<int>(s_jobs.size());
  const int64_t c_blocks = first_blocks(c_jobs);
  if (ns > 0) {
    ev = other_begin();
    ScaleJob* d_s = reinterpret_cast<ScaleJob*>(d_g + P_);
    DotJob* d_c = reinterpret_cast<DotJob*>(d_s + P_);
    char* ptrs = reinterpret_cast<char*>(d_c + P_);  // x_of, then y_of, F * nm pointers each
    const double** d_x = reinterpret_cast<const double**>(ptrs);
    double** d_y = reinterpret_cast<double**>(ptrs + static_cast<size_t>(F_) * nm_ * sizeof(double*));
    KES_CUDA(cudaMemcpyAsync(d_s, s_jobs.data(), ns * sizeof(ScaleJob), cudaMemcpyHostToDevice, s_));
    KES_CUDA(cudaMemcpyAsync(d_c, c_jobs.data(), ns * sizeof(DotJob), cudaMemcpyHostToDevice, s_));
    KES_CUDA(cudaMemcpyAsync(d_x, x_of.data(), x_of.size() * sizeof(double*), cudaMemcpyHostToDevice, s_));
    KES_CUDA(cudaMemcpyAsync(d_y, y_of.data(), y_of.size() * sizeof(double*), cudaMemcpyHostToDevice, s_));
    launch_scale_jobs(s_, d_s, ns, max_sblk);
    for (int f = 0; f < F_; ++f) {
      bool any = false;
      for (int j = 0; j < nm_; ++j) any |= x_of[static_cast<size_t>(f) * nm_ + j] != nullptr;
      if (any)
        launch_spmv_f64_meshes(c_->A, c_->cfg, s_, d_x + static_cast<size_t>(f) * nm_,
                               d_y + static_cast<size_t>(f) * nm_);
    }
    launch_mdot_jobs(s_, d_c, ns, max_k1, c_blocks, c_->partial);
    KES_CHECK_LAUNCH();
    other_end(ev);
  }
  return added;
}

// The projected matrix of process p mirrored into a full kk x kk array and its
// eigenpairs (theta ascending, clamped at 0).
void BlockSolver::projected_eig(int p, std::vector<double>& theta, std::vector<double>& Y) {
  const int kk = ms_[p].k;
  std::vector<double> Hh(static_cast<size_t>(kk) * kk, 0.0);
  KES_CUDA(cudaMemcpy2DAsync(Hh.data(), kk * sizeof(double), Hcol(p, 0), kc_ * sizeof(double), kk * sizeof(double),
                             kk, cudaMemcpyDeviceToHost, s_));
  c_->sync();
  // column i holds rows 0..i (upper triangle); mirror it into the lower triangle
  for (int i = 0; i < kk; ++i)
    for (int r = i + 1; r < kk; ++r) Hh[static_cast<size_t>(i) * kk + r] = Hh[static_cast<size_t>(r) * kk + i];
  theta.assign(kk, 0.0);
  Y.assign(static_cast<size_t>(kk) * kk, 0.0);
  if (!sym_eig(kk, Hh.data(), theta.data(), Y.data())) throw KesError{KES_ERR_CUDA};
  for (double& t : theta) t = std::max(t, 0.0);
}

// Rayleigh-Ritz (eq. projevp) and the residual acceptance (eq. res) of several processes
// at once: their projected matrices come back with one synchronisation, the small
// eigenproblems are solved on host threads, and the residual kernels run back to back
// before one more synchronisation.
void BlockSolver::project(const std::vector<int>& ps) {
  const int nps = static_cast<int>(ps.size());
  if (nps == 0) return;
  std::vector<std::vector<double>> Hs(nps), th(nps), Ys(nps);
  for (int i = 0; i < nps; ++i) {
    const int kk = ms_[ps[i]].k;
    Hs[i].assign(static_cast<size_t>(kk) * kk, 0.0);
    if (kk > 0)
      KES_CUDA(cudaMemcpy2DAsync(Hs[i].data(), kk * sizeof(double), Hcol(ps[i], 0), kc_ * sizeof(double),
                                 kk * sizeof(double), kk, cudaMemcpyDeviceToHost, s_));
  }
  c_->sync();
  std::atomic<int> next{0};
  std::atomic<bool> failed{false};
  auto worker = [&]() {
    for (int i = next++; i < nps; i = next++) {
      const int kk = ms_[ps[i]].k;
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
  const int nt = std::min(nps, std::max(1, std::min(hw, 16)));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  if (failed) throw KesError{KES_ERR_CUDA};
  std::vector<std::vector<int>> inside(nps);
  std::vector<std::vector<double>> Ysel(nps), thsel(nps), rr(nps);
  cudaEvent_t ev = other_begin();
  int64_t yo = 0, to = 0;
  for (int i = 0; i < nps; ++i) {
    const int p = ps[i];
    MeshSolve& m = ms_[p];
    const MeshInfo& mi = mesh_of(p);
    const int kk = m.k;
    m.kproj = kk;
    const double wmin = mi.wmin[p % F_], wmax = mi.wmax[p % F_];
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
    KES_CUDA(cudaMemcpyAsync(c_->Yd + yo, Ysel[i].data(), Ysel[i].size() * sizeof(double), cudaMemcpyHostToDevice,
                             s_));
    KES_CUDA(cudaMemcpyAsync(c_->thd + to, thsel[i].data(), np_in * sizeof(double), cudaMemcpyHostToDevice, s_));
    double* sc = proc_scal(c_, p);
    launch_ritz_residual(s_, Bp(p), SBp(p), np_, kk, c_->Yd + yo, c_->thd + to, np_in, c_->m64 + mi.row_off,
                         mi.n_pad, c_->partial, sc + kScal);
    KES_CHECK_LAUNCH();
    rr[i].resize(2 * np_in);
    KES_CUDA(cudaMemcpyAsync(rr[i].data(), sc + kScal, 2 * np_in * sizeof(double), cudaMemcpyDeviceToHost, s_));
    yo += static_cast<int64_t>(kk) * np_in;
    to += np_in;
  }
  other_end(ev);
  c_->sync();
  for (int i = 0; i < nps; ++i) {
    MeshSolve& m = ms_[ps[i]];
    const int kk = m.k;
    const int np_in = static_cast<int>(inside[i].size());
    for (int q = 0; q < np_in; ++q) {
      const double a = std::sqrt(std::max(rr[i][q], 0.0));
      const double den = thsel[i][q] * std::sqrt(std::max(rr[i][np_in + q], 0.0));
      const double rel = den > 0.0 ? a / den : std::numeric_limits<double>::infinity();
      m.last_rel[inside[i][q]] = rel;
      if (rel <= so_.tol) {
        m.acc_theta.push_back(thsel[i][q]);
        m.acc_rel.push_back(rel);
        m.acc_abs.push_back(a);
        m.acc_Y.insert(m.acc_Y.end(), Ysel[i].begin() + static_cast<size_t>(q) * kk,
                       Ysel[i].begin() + static_cast<size_t>(q + 1) * kk);
      }
    }
  }
}

// a mesh that asked for n_wanted pairs stops once its intervals hold that many
void BlockSolver::check_wanted() {
  if (so_.n_wanted <= 0) return;
  for (int j = 0; j < nm_; ++j) {
    int got = 0;
    for (int f = 0; f < F_; ++f) got += static_cast<int>(ms_[j * F_ + f].acc_theta.size());
    if (got >= so_.n_wanted)
      for (int f = 0; f < F_; ++f) ms_[j * F_ + f].done = true;
  }
}

// The start block: the g start vectors of each process, M-orthonormalised in order.
void BlockSolver::start(const double* R0, int32_t mem) {
  cudaEvent_t ev = other_begin();
  block_in(c_, R0, b_, mem, NB_, c_->stage_in);
  launch_unpack_block(s_, c_->stage_in, NB_, c_->Wc, np_);
  KES_CHECK_LAUNCH();
  other_end(ev);
  for (int jj = 0; jj < b_; ++jj) orthogonalise(jj);
  for (int p = 0; p < P_; ++p)
    if (ms_[p].k == 0) ms_[p].done = ms_[p].breakdown = true;
}

// Block steps until every process is done: filter the g newest basis vectors of each
// process in one trajectory (Algorithm 2.5 filters the newest one), orthogonalise the
// filtered columns into the bases, project the processes whose check is due; then the
// final projection of every process whose basis grew since its last one.
void BlockSolver::krylov() {
  std::vector<int> next_check(P_, so_.check_every);
  std::vector<int32_t> colsel(static_cast<size_t>(nm_) * NB_, -1);
  for (;;) {
    bool any = false;
    std::fill(colsel.begin(), colsel.end(), -1);
    for (int p = 0; p < P_; ++p) {
      MeshSolve& m = ms_[p];
      if (m.done || m.k >= kmax_) continue;
      any = true;
      const int j = p / F_, f = p % F_;
      for (int i = 0; i < g_; ++i) {
        const int col = m.k - g_ + i;
        colsel[j * NB_ + f * g_ + i] = col >= 0 ? static_cast<int32_t>(f * kc_ + col) : -1;
      }
    }
    if (!any) break;
    KES_CUDA(cudaMemcpyAsync(c_->colsel, colsel.data(), colsel.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s_));
    launch_pack_basis(s_, c_->B, np_, c_->colsel, c_->slice_mesh, c_->stage_in, NB_, np_);
    KES_CHECK_LAUNCH();
    run_filter(c_, NB_, c_->opts.precision == KES_PREC_FP64, cpt_);  // stage_in -> stage_out
    steps_ += c_->L;
    launch_unpack_block(s_, c_->stage_out, NB_, c_->Wc, np_);
    KES_CHECK_LAUNCH();
    std::vector<int> added(P_, 0);
    for (int jj = 0; jj < b_; ++jj) {
      std::vector<char> a = orthogonalise(jj);
      for (int p = 0; p < P_; ++p) added[p] += a[p];
    }
    std::vector<int> due;
    for (int p = 0; p < P_; ++p) {
      MeshSolve& m = ms_[p];
      if (m.done) continue;
      if (added[p] == 0 && m.k < kmax_) {  // the whole block was dependent: invariant subspace
        m.done = m.breakdown = true;
        continue;
      }
      if (m.k >= next_check[p] && m.k < kmax_) {
        while (next_check[p] <= m.k) next_check[p] += so_.check_every;
        due.push_back(p);
      }
    }
    project(due);
    check_wanted();
  }
  std::vector<int> due;
  for (int p = 0; p < P_; ++p)
    if (ms_[p].kproj != ms_[p].k) due.push_back(p);
  project(due);
}

// Sweeps of filtered subspace iteration (Sec. 4 mentions the fixed-dimension, FEAST-like
// use of the filter): X <- C X, M-orthonormalise, Rayleigh-Ritz, residuals. After the
// Krylov phase (refinement) the sweeps filter in-interval Ritz vectors with the FP64
// kernels; in the fixed-dimension mode (X0) they filter in the context's precision and
// keep every Ritz vector. With F intervals the columns of a refinement block are grouped
// per interval like those of the Krylov blocks.
void BlockSolver::refine(int32_t mem) {
  const int NBr = F_ > 1 ? NB_ : c_->NBcap;  // columns of one refinement filter call
  const int gr = F_ > 1 ? g_ : NBr;          // of them per interval
  const bool sweep_fp64 = X0_ ? c_->opts.precision == KES_PREC_FP64 : true;
  // FP32-form contexts may take the sweeps' filter in FP32 pairs instead (same recurrence and
  // weights, a ~48-bit significand on the FP32 units)
  const bool sweep_x2 = so_.refine_precision == KES_REFINE_F32X2 && c_->opts.precision == KES_PREC_FP32;
  // the Ritz vectors a sweep filters: all of them (fixed-dimension mode), or those with Ritz
  // values in the interval plus the refine_extra nearest outside it (a buffer, as FEAST
  // keeps more vectors than eigenvalues wanted)
  std::vector<std::vector<char>> keepq(P_);
  auto select = [&](int p) {
    const MeshSolve& m = ms_[p];
    const int kk = static_cast<int>(m.last_rel.size());
    keepq[p].assign(kk, 0);
    std::vector<std::pair<double, int>> outside;
    const MeshInfo& mi = mesh_of(p);
    const double wmin = mi.wmin[p % F_], wmax = mi.wmax[p % F_];
    for (int q = 0; q < kk; ++q) {
      if (X0_ != nullptr || !std::isnan(m.last_rel[q])) {
        keepq[p][q] = 1;
      } else if (so_.refine_extra > 0) {
        const double om = std::sqrt(m.last_theta[q]);
        outside.emplace_back(om < wmin ? wmin - om : om - wmax, q);
      }
    }
    std::sort(outside.begin(), outside.end());
    for (int e = 0; e < so_.refine_extra && e < static_cast<int>(outside.size()); ++e) keepq[p][outside[e].second] = 1;
  };
  auto keep = [&](int p, int q) { return keepq[p][q] != 0; };
  for (int sweep = 0; sweep < so_.refine_sweeps; ++sweep) {
    const bool from_x0 = X0_ && sweep == 0;
    if (!from_x0)
      for (int p = 0; p < P_; ++p) select(p);
    std::vector<int> pcount(P_, 0);
    std::vector<int64_t> xoff(F_ + 1, 0);  // interval f uses columns xoff[f] .. of Xd (meshes share them)
    int rounds = 0;
    for (int p = 0; p < P_; ++p) {
      if (from_x0) pcount[p] = p0_;
      else
        for (size_t q = 0; q < ms_[p].last_rel.size(); ++q) pcount[p] += keep(p, static_cast<int>(q)) ? 1 : 0;
      rounds = std::max(rounds, (pcount[p] + gr - 1) / gr);
    }
    for (int f = 0; f < F_; ++f) {
      int mx = 0;
      for (int j = 0; j < nm_; ++j) mx = std::max(mx, pcount[j * F_ + f]);
      xoff[f + 1] = xoff[f] + mx;
    }
    if (xoff[F_] == 0) break;
    const size_t need = static_cast<size_t>(xoff[F_]) * np_;
    if (need > c_->Xd_cap) {
      c_->dfree(c_->Xd);
      c_->Xd = c_->dalloc_n<double>(need);
      c_->Xd_cap = need;
    }
    KES_CUDA(cudaMemsetAsync(c_->Xd, 0, need * sizeof(double), s_));
    if (from_x0) {  // the caller's vectors, one column at a time into the padded row order
      for (int q = 0; q < p0_; ++q) {
        const double* src = X0_ + static_cast<int64_t>(q) * c_->n;
        if (mem == KES_MEM_HOST) {
          KES_CUDA(cudaMemcpyAsync(c_->tmp_user, src, static_cast<size_t>(c_->n) * sizeof(double),
                                   cudaMemcpyHostToDevice, s_));
          src = c_->tmp_user;
        }
        launch_gather_rows(s_, src, c_->n, 1, c_->row_src, c_->n, c_->Xd + static_cast<int64_t>(q) * np_, 1, np_);
      }
      KES_CHECK_LAUNCH();
    }
    // Ritz vectors (all of them, or those of in-interval Ritz values): X = B y_q
    for (int p = 0; p < P_ && !from_x0; ++p) {
      if (pcount[p] == 0) continue;
      MeshSolve& m = ms_[p];
      const MeshInfo& mi = mesh_of(p);
      const int kk = m.k;
      std::vector<double> theta, Y, Ysel;
      projected_eig(p, theta, Y);
      for (int q = 0; q < kk; ++q)
        if (keep(p, q))
          Ysel.insert(Ysel.end(), Y.begin() + static_cast<size_t>(q) * kk, Y.begin() + static_cast<size_t>(q + 1) * kk);
      KES_CUDA(cudaMemcpyAsync(c_->Yd, Ysel.data(), Ysel.size() * sizeof(double), cudaMemcpyHostToDevice, s_));
      launch_gemm_bx(s_, Bp(p), np_, kk, c_->Yd, pcount[p], c_->Xd + xoff[p % F_] * np_ + mi.row_off, np_, mi.n_pad);
      KES_CHECK_LAUNCH();
      c_->sync();  // Yd is reused by the next process
    }
    // filter them, a block of NBr columns at a time, into fresh bases
    for (int p = 0; p < P_; ++p) {
      want_[p] = pcount[p] > 0;
      if (want_[p]) {
        ms_[p].k = 0;
        ms_[p].done = false;
      }
    }
    std::vector<int32_t> csel(static_cast<size_t>(nm_) * NBr, -1);
    for (int r = 0; r < rounds; ++r) {
      std::fill(csel.begin(), csel.end(), -1);
      for (int p = 0; p < P_; ++p) {
        const int j = p / F_, f = p % F_;
        for (int i = 0; i < gr; ++i) {
          const int q = r * gr + i;
          if (q < pcount[p]) csel[j * NBr + f * gr + i] = static_cast<int32_t>(xoff[f] + q);
        }
      }
      KES_CUDA(cudaMemcpyAsync(c_->colsel, csel.data(), csel.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s_));
      launch_pack_basis(s_, c_->Xd, np_, c_->colsel, c_->slice_mesh, c_->stage_in, NBr, np_);
      KES_CHECK_LAUNCH();
      const int Lr = so_.refine_L > 0 && so_.refine_L < c_->L ? so_.refine_L : c_->L;
      run_filter(c_, NBr, sweep_fp64, cpt_, Lr, sweep_x2);
      refine_steps_ += Lr;
      launch_unpack_block(s_, c_->stage_out, NBr, c_->Wc, np_);
      KES_CHECK_LAUNCH();
      for (int jj = 0; jj < NBr; ++jj) {
        bool any = false;
        for (int j = 0; j < nm_; ++j) {
          const int p = owner(j, jj);
          if (p < 0) continue;
          want_[p] = csel[j * NBr + jj] >= 0;
          any |= want_[p] != 0;
        }
        if (any) orthogonalise(jj);
      }
    }
    std::vector<int> due;
    for (int p = 0; p < P_; ++p) {
      if (pcount[p] > 0) due.push_back(p);
      want_[p] = 1;
    }
    project(due);
  }
}

// The pairs of each mesh's processes merged in ascending theta, with the accepted Ritz
// vectors when asked for. Returns whether any process broke down.
bool BlockSolver::results(std::vector<kes_result*>& res) {
  bool any_breakdown = false;
  for (int j = 0; j < nm_; ++j) {
    const MeshInfo& mi = c_->meshes[j];
    kes_result* r = res[j];
    struct Pair {
      double theta;
      int f, q;
    };
    std::vector<Pair> pairs;
    std::vector<double> ritz_th, ritz_rel;
    int k_used = 0;
    bool brk = false;
    for (int f = 0; f < F_; ++f) {
      const MeshSolve& m = ms_[j * F_ + f];
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
      const MeshSolve& m = ms_[j * F_ + pairs[t].f];
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
    r->time_steps = steps_;
    r->refine_steps = refine_steps_;
    r->omega2 = hdup(th);
    r->omega = hdup(om);
    r->rel_res = hdup(rel);
    r->abs_res = hdup(ab);
    r->interval = hdup(iv);
    r->ritz_omega2 = hdup(ritz_th);
    r->ritz_rel_res = hdup(ritz_rel);
    if (so_.want_vectors && np_acc > 0) {
      const size_t need = static_cast<size_t>(np_acc) * np_;
      if (need > c_->Xd_cap) {
        c_->dfree(c_->Xd);
        c_->Xd = c_->dalloc_n<double>(need);
        c_->Xd_cap = need;
      }
      KES_CUDA(cudaMemsetAsync(c_->Xd, 0, need * sizeof(double), s_));
      // interval f's accepted vectors go to columns xo[f] .. of Xd
      std::vector<int> xo(F_ + 1, 0);
      for (int f = 0; f < F_; ++f) {
        const MeshSolve& m = ms_[j * F_ + f];
        const int cnt = static_cast<int>(m.acc_theta.size());
        xo[f + 1] = xo[f] + cnt;
        if (cnt == 0) continue;
        KES_CUDA(cudaMemcpyAsync(c_->Yd, m.acc_Y.data(), m.acc_Y.size() * sizeof(double), cudaMemcpyHostToDevice, s_));
        launch_gemm_bx(s_, Bp(j * F_ + f), np_, m.k, c_->Yd, cnt, c_->Xd + static_cast<int64_t>(xo[f]) * np_ + mi.row_off,
                       np_, mi.n_pad);
        KES_CHECK_LAUNCH();
        c_->sync();  // Yd is reused by the next interval
      }
      r->vectors = static_cast<double*>(std::malloc(static_cast<size_t>(np_acc) * mi.n * sizeof(double)));
      if (!r->vectors) throw std::bad_alloc();
      // scatter each Ritz vector to the caller's order and keep this mesh's rows
      for (int t = 0; t < np_acc; ++t) {
        const int64_t col = xo[pairs[t].f] + pairs[t].q;
        launch_scatter_rows(s_, c_->Xd + col * np_, 1, 1, c_->row_src, c_->n, c_->tmp_user, c_->n, np_);
        KES_CHECK_LAUNCH();
        KES_CUDA(cudaMemcpyAsync(r->vectors + static_cast<size_t>(t) * mi.n, c_->tmp_user + mi.src_off,
                                 mi.n * sizeof(double), cudaMemcpyDeviceToHost, s_));
      }
      c_->sync();
    }
  }
  c_->sync();
  return any_breakdown;
}

}  // namespace

kes_status block_solve_impl(kes_ctx* c, const double* R0, int b, int32_t mem, const kes_solve_opts& so,
                            kes_result** out, const double* X0, int p0) {
  const int nm = c->n_mesh();
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
    ensure_krylov(c, so.kmax, c->F);
    BlockSolver solver(c, b, so, X0, p0);
    if (!X0) {
      solver.start(R0, mem);
      solver.krylov();
    }
    solver.refine(mem);
    return solver.results(res) ? KES_INFO_INVARIANT_SUBSPACE : KES_OK;
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

}  // namespace kes
