// Internal declarations of the kes library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "kes.h"

namespace kes {

constexpr int kSliceC = 32;  // SELL slice height = warp width

// ---------------------------------------------------------------- host math
void alpha_table(double wmin, double wmax, double tau, int L, double* alpha);
void filter_response(double wmin, double wmax, double tau, int L, const double* omega, int64_t k,
                     double* beta);
void alpha_gaussian(double center, double sigma, double tau, int L, double* alpha);
void alpha_triangle(double center, double half_width, double tau, int L, double* alpha);
void weights_response(const double* alpha, double tau, int L, const double* omega, int64_t k, double* beta);
// Symmetric eigensolver for the projected problem: Householder tridiagonalisation
// followed by implicit QR steps with Wilkinson shifts. A is k x k col-major (lower
// triangle read), w ascending, V (optional) orthonormal eigenvectors col-major.
bool sym_eig(int k, const double* A, double* w, double* V);

// ---------------------------------------------------------------- SELL-C-sigma
struct SellHost {
  int64_t n = 0, n_slices = 0, nnz = 0, nnz_pad = 0;
  std::vector<int64_t> slice_ptr;  // [n_slices+1] element offsets, multiples of 32
  std::vector<int32_t> col;        // [nnz_pad], entry (lane, k) of slice s at slice_ptr[s] + 32k + lane
  std::vector<double> val;         // [nnz_pad], 0 in padding
  std::vector<int32_t> perm;       // new row i = old row perm[i]; empty = identity
};
// Rows are sorted by decreasing length inside windows of `sigma` rows (sigma = 1
// keeps the order); the permutation is applied symmetrically so that every
// vector lives in the permuted order. Padding entries repeat the row's own index
// with value 0 (phantom rows past n use column n-1).
SellHost build_sell(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val, int sigma);

// ---------------------------------------------------------------- kernels
struct SellDev {
  int64_t n = 0, n_pad = 0, n_slices = 0;
  const int64_t* slice_ptr = nullptr;
  const int32_t* col = nullptr;
  // compact index of the step kernels: column - row of every stored entry as 16 bits,
  // when all of them fit (null otherwise); the same columns as `col`
  const int16_t* dcol = nullptr;
  // pair layout of the single-vector steps: a lane's entries 2k and 2k+1 adjacent, at
  // slice_ptr2[s] + 64 (k / 2) + 2 lane + k % 2, odd slice widths padded with one zero entry
  // per lane (difference 0, skipped by the row sums); values val32p / val64p, differences
  // dcolp. Null where not built; val64p is built only where fold2 is set.
  const int64_t* slice_ptr2 = nullptr;
  const float* val32p = nullptr;
  const double* val64p = nullptr;
  const int16_t* dcolp = nullptr;
  const double* val64 = nullptr;
  const float* val32 = nullptr;
  // the FP64 step values (val64, val64p) hold A + 2I: the leapfrog's 2 u_n folded into the
  // diagonal, so a row sum seeds with -u_{n-1} alone (FP32 values never hold it)
  int fold2 = 0;
  // mesh of each slice when several meshes are stacked block-diagonally (null: one mesh).
  // Weight tables are indexed (mesh * F + f) * (L + 1) + n.
  const int32_t* slice_mesh = nullptr;
};

struct LaunchCfg {
  int grid_step = 0;   // blocks of the step / SpMV kernels (grid-stride over slices)
  int block_step = 256;
  int n_sm = 152;
  int variant = 0;     // step-kernel launch shape (load batch, register cap), see step_variant_count
  int grid_blk = 0;    // blocks of the block (SpMM) step kernels
  int variant_blk = 0; // their launch shape (register cap), see blk_variant_count
};

// One fused leapfrog step, FP64 (Sec. 2.3, eq. 2stepmethod + eq. disc_filtercoeff), on the
// values of A = -tau^2 M^{-1} S (see launch_scale_values):
//   out = (2 x - prev) + A g;   acc_f += alpha_f[step+1] * out   (f < F)
// (A.fold2: out = -prev + (A + 2I) x, the same sum with the 2 x in the diagonal values.)
// g = x for the leapfrog; g = the stage v = x + A x / 12 (launch_stage4_*) for the
// fourth-order scheme.
// first: prev = x and acc_f = alpha_f[0] * x + alpha_f[1] * out.
// x, prev, out, acc: length n_pad; acc_f at acc + f * acc_stride; alpha of mesh m, table f at
// alpha + (m * F + f) * (L+1). last: the state of the final step is not stored;
// flag[0] |= 1 if any acc entry is not finite. nterm / init: the accumulation of this step
// (acc_plan; the last step needs nterm >= 1).
void launch_step_f64(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, bool first,
                     const double* x, const double* g, const double* prev, double* out,
                     double* acc, int64_t acc_stride, int F, const double* alpha, int L, int step,
                     bool last, int nterm, bool init, int* flag);

// FP32 form: values/state FP32, accumulator as an unevaluated FP32 sum (s + c) kept by
// error-free transformations; alpha as FP32 pairs (hi + lo). last: writes acc64 = s + c in FP64.
void launch_step_f32(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, bool first, bool last,
                     const float* x, const float* g, const float* prev, float* out, float* acc_s,
                     float* acc_c, double* acc64, int64_t acc_stride, int F, const float* alpha_hi,
                     const float* alpha_lo, int L, int step, int nterm, int* flag);
// FP32 start over n_pad x nb row-major values: x32 = (float) r64; s_f = fl(alpha_f[0] r),
// c_f = alpha_f[0] r - s_f (rounded), with the weight table of each row's mesh (cpt > 0:
// column j has one accumulator, with table j / cpt).
void launch_init_f32(cudaStream_t st, const SellDev& A, int nb, const double* r64, float* x32, float* acc_s,
                     float* acc_c, int64_t acc_stride, int F, const double* alpha64, int L, int cpt);

// Block step (SpMM form) for NB in {2, 4, 8} columns, row-major n_pad x NB state
// (row i's NB values contiguous). Same arithmetic per column as the single-vector
// kernels; acc_stride = n_pad * NB elements per accumulator set. cpt = 0: every column
// accumulates with all F weight tables; cpt > 0: column j only with table j / cpt (the
// columns of several intervals share the matrix stream). nterm = 0: the step leaves the
// accumulators alone; 1-3: it adds the last nterm of alpha_{s-1} u_{s-1}, alpha_s u_s,
// alpha_{s+1} u_{s+1} in that order (step s computes u_{s+1}; the last step needs
// nterm >= 1). init (FP64): the accumulator starts at the first of them (the FP32 form's
// accumulators start from launch_init_f32). acc_plan gives the schedule.
void launch_step_blk_f64(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, int NB, bool first, bool last,
                         const double* x, const double* g, const double* prev, double* out, double* acc,
                         int64_t acc_stride, int F, const double* alpha, int L, int step, int cpt, int nterm,
                         bool init, int* flag);
void launch_step_blk_f32(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, int NB, bool first, bool last,
                         const float* x, const float* g, const float* prev, float* out, float* acc_s, float* acc_c,
                         double* acc64, int64_t acc_stride, int F, const float* alpha_hi, const float* alpha_lo,
                         int L, int step, int cpt, int nterm, int* flag);
// Block step in FP32 pairs (hi + lo, double-float arithmetic) for NB in {2, 4, 8} columns:
// state rows of NB float2 (n_pad x NB row-major), step values val2 (the FP64 step values split,
// SELL order of val64), the compensated FP32 accumulators and weights of the FP32 form;
// nterm as for launch_step_blk_f32.
void launch_step_x2(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, int NB, bool first, bool last,
                    const float2* val2, const float2* x, const float2* prev, float2* out, float* acc_s, float* acc_c,
                    double* acc64, int64_t acc_stride, int F, const float* alpha_hi, const float* alpha_lo, int L,
                    int step, int cpt, int nterm, int* flag);
// Start of a filter application in FP32 pairs: x2 = r64 split, accumulators as launch_init_f32.
void launch_init_x2(cudaStream_t st, const SellDev& A, int nb, const double* r64, float2* x2, float* acc_s,
                    float* acc_c, int64_t acc_stride, int F, const double* alpha64, int L, int cpt);
// v2[i] = (fl(v[i]), fl(v[i] - fl(v[i]))) for count values
void launch_split_values(cudaStream_t st, int64_t count, const double* v, float2* v2);
// Accumulation schedule of a filter application of `steps` fused steps (single-vector and
// block kernels): the weighted terms reach the accumulators every third step and at the last. next is the index of the first
// term not yet added (0 for the FP64 form, 1 for the FP32 form, whose initialisation adds
// alpha_0 u_0); returns the step's nterm and advances next.
inline int acc_plan(int s, int steps, int& next, bool& init) {
  const int pending = s + 2 - next;  // terms u_next .. u_{s+1}
  if (pending < 3 && s != steps - 1) return 0;
  init = next == 0;
  next = s + 2;
  return pending;
}
// Stage of the fourth-order modified-equation leapfrog: v = x + A x / 12 over NB row-major
// columns (NB in {1, 2, 4, 8}; n_pad x NB).
void launch_stage4_f64(const SellDev& A, int n_sm, cudaStream_t st, int NB, const double* x, double* v);
void launch_stage4_f32(const SellDev& A, int n_sm, cudaStream_t st, int NB, const float* x, float* v);
int blk_variant_count();
int blk_blocks_per_sm(bool fp32, int NB, int variant, int block);

// Row-major block <-> user / basis layouts.
//   gather_rows: dst[i*NB + j] = src[j*ld_src + row_src[i]] for j < ncols and row_src[i] >= 0, else 0
//   scatter_rows: dst[j*ld_dst + row_src[i]] = src[i*NB + j] for j < ncols, row_src[i] >= 0
//   (row_src null: the identity for i < n_valid)
void launch_gather_rows(cudaStream_t st, const double* src, int64_t ld_src, int ncols, const int32_t* row_src,
                        int64_t n_valid, double* dst, int NB, int64_t n_pad);
void launch_scatter_rows(cudaStream_t st, const double* src, int NB, int ncols, const int32_t* row_src,
                         int64_t n_valid, double* dst, int64_t ld_dst, int64_t n_pad);
//   pack_basis: stage[i*NB + j] = B[colsel[mesh(i)*NB + j] * ldb + i] (colsel < 0: 0)
//   unpack_block: Wc[j*n_pad + i] = stage[i*NB + j]
void launch_pack_basis(cudaStream_t st, const double* B, int64_t ldb, const int32_t* colsel,
                       const int32_t* slice_mesh, double* stage, int NB, int64_t n_pad);
void launch_unpack_block(cudaStream_t st, const double* stage, int NB, double* Wc, int64_t n_pad);

// Launch-shape variants of the step kernels (same arithmetic, different load batch and
// register cap) and the resident blocks per SM of one variant (occupancy calculator);
// the step grid is n_sm * that, so that the grid-stride loop runs in one wave.
int step_variant_count();
int step_blocks_per_sm(bool fp32, int variant, int block);

// Step values A = -tau^2 M^{-1} S from the values of S (A.val64) and tau^2/m per row:
// out64[e] = -tau2m[row(e)] * val64[e] and/or out32[e] = (float) of the same (either may be null).
// fold2: out64 and out64p get 2 added at each row's first entry at its own column (A + 2I);
// the caller has checked that every row has one.
void launch_scale_values(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, const double* tau2m,
                         double* out64, float* out32, double* out64p,
                         float* out32p,  // out64p / out32p: pair layout (A.slice_ptr2)
                         bool fold2);

// y = dscale .* (S x) (dscale may be null) in FP64.
void launch_spmv_f64(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, const double* x,
                     const double* dscale, double* y);

// Sets flag[0] = 1 if any of v[0..n) is not finite.
void launch_check_finite(cudaStream_t st, const double* v, int64_t n, int* flag);

// Batched forms of the Gram-Schmidt kernels: one launch serves every process (mesh and
// interval) of a block step. A job is one process's part; it is reduced through the same
// number of row blocks as the single launch for its rows would use (rows_for_dot), so the
// results are bit for bit those of the separate launches.
struct DotJob {        // out[j] = sum_i B[j * ldb + i] * (w ? w[i] : 1) * v[i], j < k
  const double* B;
  const double* v;
  const double* w;
  double* out;
  int64_t n;
  int64_t ldb;
  int64_t poff;        // offset of this job's k * nblk partial sums in `partial`
  int64_t first;       // its first block of the launch (set by launch_mdot_jobs' caller: prefix sums)
  int k;
  int nblk;
};
struct GemvJob {       // v -= B h (k columns)
  double* v;
  const double* B;
  const double* h;
  int64_t n;
  int64_t ldb;
  int64_t first;       // its first block of the launch
  int k;
  int nblk;
};
// Blocks a job takes in a batched launch (the launch's grid is the sum over its jobs).
inline int64_t dot_job_blocks(const DotJob& j) { return j.nblk; }
inline int64_t gemv_job_blocks(const GemvJob& j) { return j.nblk; }
struct ScaleJob {      // dst = v / sqrt(nrm2[0])
  const double* v;
  const double* nrm2;
  double* dst;
  int64_t n;
};
int dot_blocks(int64_t n);   // row blocks of a batched inner-product job over n rows
int gemv_blocks(int64_t n);  // row blocks of launch_gemv_sub for n rows
// total_blocks: sum of dot_job_blocks / gemv_job_blocks over the jobs, whose `first` fields
// hold the prefix sums in job order.
void launch_mdot_jobs(cudaStream_t st, const DotJob* jobs, int njobs, int max_k, int64_t total_blocks,
                      double* partial);
void launch_gemv_sub_jobs(cudaStream_t st, const GemvJob* jobs, int njobs, int max_k, int64_t total_blocks);
void launch_scale_jobs(cudaStream_t st, const ScaleJob* jobs, int njobs, int max_nblk);
// S x for the slices of every mesh at once, each with its own vectors: x_of[mesh] (global
// row indexing) and y_of[mesh]; a mesh with a null x_of is skipped.
void launch_spmv_f64_meshes(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, const double* const* x_of,
                            double* const* y_of);

// h_j = sum_i B[j*ldb + i] * w[i] * v[i] for j < k (w may be null); deterministic two-pass
// reduction through `partial` (size >= k * kDotBlocks); result written to h (device).
constexpr int kDotBlocks = 608;
// Largest basis (Krylov dimension per process) the projection kernels take: their shared
// memory holds k x 8 doubles, within the 227 KB a GB300 block may opt in to.
constexpr int kMaxProjected = 3584;
void launch_mdot(cudaStream_t st, const double* B, int64_t ldb, int k, const double* v, const double* w,
                 int64_t n, double* partial, double* h);
// v[i] -= sum_j B[j*ldb + i] * h[j], j < k
void launch_gemv_sub(cudaStream_t st, double* v, const double* B, int64_t ldb, int k, const double* h,
                     int64_t n);
// dst[i] = v[i] / sqrt(nrm2[0]) (dst2 may be null: second copy)
void launch_scale_rsqrt(cudaStream_t st, const double* v, const double* nrm2, double* dst, double* dst2,
                        int64_t n);
// residuals of Ritz pairs: for j < p, x_j = B Y_j, sx_j = SB Y_j (k terms);
// out[j] = ||sx_j - theta_j m x_j||_2^2, out[p + j] = ||m x_j||_2^2
void launch_ritz_residual(cudaStream_t st, const double* B, const double* SB, int64_t ldb, int k,
                          const double* Y, const double* theta, int p, const double* m, int64_t n,
                          double* partial, double* out);
// X[:, j] = B Y_j, j < p (X: ldx-strided columns)
void launch_gemm_bx(cudaStream_t st, const double* B, int64_t ldb, int k, const double* Y, int p,
                    double* X, int64_t ldx, int64_t n);
// dst[i] = src[perm[i]] (gather into permuted order) / dst[perm[i]] = src[i] (scatter back)
void launch_permute(cudaStream_t st, const double* src, double* dst, const int32_t* perm, int64_t n,
                    bool gather);
// dst[i] = src[i] * s
void launch_scale(cudaStream_t st, const double* src, double s, double* dst, int64_t n);

extern thread_local int64_t g_launches;  // kernels launched by this thread (stats)

}  // namespace kes
