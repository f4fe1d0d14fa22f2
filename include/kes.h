/*
 * kes.h -- C ABI of the filtered time-domain Krylov eigensolver for GB300.
 *
 * Method: Nannen & Wess, "A Krylov Eigenvalue Solver Based on Filtered Time
 * Domain Solutions" (arXiv:2402.08515), Sec. 2. The library finds eigenpairs
 * (omega^2, v) of S v = omega^2 M v (eq. def:basisMatrixEVP) with omega in a
 * chosen interval [omega_min, omega_max], for a sparse symmetric positive
 * semi-definite S and a lumped (diagonal, positive) M (Remark 2.1).
 *
 * Conventions shared by every entry point:
 *   - Every function returns a kes_status (0 = success); no C++ exception and
 *     no CUDA error crosses the ABI. kes_strerror() names a status.
 *   - Arrays are plain pointers. "host" pointers are ordinary CPU memory,
 *     "device" pointers are CUDA global memory on the context's device.
 *     A `mem` argument (KES_MEM_HOST / KES_MEM_DEVICE) says which.
 *   - Blocks of vectors are n x b column-major: vector j starts at j * n.
 *   - The library copies every input it keeps; the caller keeps ownership of
 *     what it passes. Results returned through kes_result are owned by the
 *     library and released with kes_result_free().
 *   - All GPU work is issued on the context's stream (kes_opts.stream). Calls
 *     that return host data synchronise that stream; kes_filter_apply with
 *     device pointers does not (use kes_sync).
 *   - Indices are 0-based. Real symmetric input only; Dirichlet dofs must be
 *     eliminated by the caller.
 */
#ifndef KES_H
#define KES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kes_ctx kes_ctx;

typedef enum kes_status {
  KES_OK = 0,
  KES_INFO_INVARIANT_SUBSPACE = 1, /* Krylov breakdown: an invariant subspace was found (Algorithm 2.5, "exact eigenspace found") */
  KES_ERR_ARG = -1,                /* invalid argument (null pointer, size, range, ordering) */
  KES_ERR_MASS = -2,               /* a lumped mass entry is <= 0 or not finite */
  KES_ERR_UNSTABLE = -3,           /* CFL violated (tau * omega_max >= 2, or 2 sqrt(3) for the fourth-order
                                      stepper) or the time stepping produced Inf/NaN */
  KES_ERR_CUDA = -4,               /* a CUDA runtime call failed */
  KES_ERR_OOM = -5,                /* device or host allocation failed */
  KES_ERR_TIMEOUT = -6,            /* a bounded device-side wait gave up (reserved: no kernel of this
                                      library waits on another thread block) */
  KES_ERR_STATE = -7,              /* call out of order (e.g. filter not set) */
  KES_ERR_UNSUPPORTED = -8         /* option combination not implemented */
} kes_status;

/* Time stepper of the filter (Remark 2.4: any explicit scheme diagonalised by the
   eigenvectors keeps Lemma 2.3, with its own scalar recurrence q_l). */
enum kes_stepper {
  KES_STEPPER_LEAPFROG = 0,  /* eq. (2stepmethod): y_{l+1} = 2 y_l - y_{l-1} - tau^2 K y_l, K = M^{-1} S;
                                q_{l+1} = (2 - x) q_l - q_{l-1}, x = tau^2 omega^2; stable for tau omega < 2 */
  KES_STEPPER_LEAPFROG4 = 1  /* fourth-order modified equation: ... + (tau^4 / 12) K^2 y_l (two sparse products
                                per step); q_{l+1} = (2 - x + x^2 / 12) q_l - q_{l-1}; stable for
                                tau omega <= 2 sqrt(3), phase error O((omega tau)^5) */
};

enum kes_precision {
  KES_PREC_FP64 = 0, /* FP64 matrix values, state and accumulation */
  KES_PREC_FP32 = 1  /* FP32 matrix values and leapfrog state, compensated (two-sum) FP32 accumulation;
                        orthogonalisation, Rayleigh-Ritz and residuals stay FP64 */
};

enum kes_mem { KES_MEM_DEVICE = 0, KES_MEM_HOST = 1 };

/* Options of kes_create. Initialise with kes_opts_default(). */
typedef struct kes_opts {
  int32_t precision;   /* enum kes_precision */
  int32_t sell_sigma;  /* SELL-C-sigma sorting window in rows (slices are C = 32 rows); 1 keeps the row order */
  int32_t use_graph;   /* 1: the L time steps of a filter application replay as one CUDA graph; 0: plain launches */
  int32_t block_b;     /* largest number of start vectors filtered together (columns of kes_filter_apply and
                          the block size of kes_block_krylov_solve), 1..8; blocks of 2, 4 or 8 columns run
                          as one SpMM step (row-major state), other sizes are padded to the next of them */
  int32_t autotune;    /* 1: kes_create times every launch shape of the step kernel on this matrix and keeps the
                          fastest (results do not depend on the choice); 0: use step_variant */
  int32_t step_variant; /* launch shape used when autotune is 0 (0 .. number of shapes - 1) */
  void* stream;        /* cudaStream_t for every launch; NULL: the context creates its own non-blocking stream */
  /* Optional device allocator (e.g. a framework's caching allocator). Both NULL: cudaMalloc / cudaFree. */
  void* (*dev_alloc)(size_t bytes, void* user);
  void (*dev_free)(void* ptr, size_t bytes, void* user);
  void* alloc_user;
  int32_t stepper;     /* enum kes_stepper (default KES_STEPPER_LEAPFROG) */
  int32_t blk_variant; /* launch shape of the block (SpMM) step kernel when autotune is 0 */
  int32_t compact_cols; /* 1 (default): the step kernels read each stored entry's column as the 16-bit
                           difference column - row when every entry's fits (2 bytes instead of 4: tensor
                           grids up to about 180 x 180 nodes per plane), else as int32; 0: always int32.
                           Results are the same either way. */
} kes_opts;

/* Options of kes_krylov_solve. Initialise with kes_solve_opts_default(). */
typedef struct kes_solve_opts {
  int32_t kmax;         /* Krylov dimension: number of basis vectors b_0..b_{kmax-1} (kmax-1 filter applications);
                           at most 3584 (KES_ERR_UNSUPPORTED above: the projection kernels hold kmax x 8
                           coefficients in one block's shared memory) */
  int32_t check_every;  /* solve the projected problem every this many new basis vectors (and at the end) */
  int32_t n_wanted;     /* stop as soon as this many pairs are accepted (0: run to kmax) */
  int32_t want_vectors; /* 1: return the accepted Ritz vectors B y (host, n x n_pairs col-major) */
  double tol;           /* acceptance: rel_res = ||S x - theta M x||_2 / (theta ||M x||_2) <= tol */
  int32_t refine_sweeps; /* after the Krylov phase: sweeps of filtered subspace iteration on the
                            in-interval Ritz vectors (X <- C X with the FP64 step kernels, or in FP32
                            pairs per refine_precision, then FP64 Gram-Schmidt and Rayleigh-Ritz, Sec. 4);
                            lifts FP32-form pairs to FP64 residuals. 0: none */
  int32_t refine_L;      /* leapfrog steps of the refinement filter: the first refine_L + 1 weights of the
                            installed tables, i.e. the same interval with end time refine_L * tau
                            (eq. weightf does not depend on T); 0 or >= L: L */
  int32_t refine_extra;  /* the refinement sweeps also filter this many Ritz vectors whose Ritz values lie
                            nearest outside the interval (a buffer; 0: the in-interval ones only) */
  int32_t refine_precision; /* arithmetic of the refinement sweeps' filter (enum kes_refine_precision):
                            KES_REFINE_FP64 (default) or KES_REFINE_F32X2; the latter in contexts of the
                            FP32 form with the leapfrog stepper and block_b >= 2 (KES_ERR_UNSUPPORTED
                            otherwise); contexts of the FP64 form filter in FP64 either way */
} kes_solve_opts;

/* Arithmetic of the refinement sweeps' filter steps. KES_REFINE_F32X2 keeps step values,
   states and row sums as unevaluated sums hi + lo of two FP32 numbers (double-float
   arithmetic: error-free products by FMA and Knuth's two-sum, a significand of about 48
   bits) on the FP32 units, with the compensated FP32 accumulator of the FP32 form; on GB300,
   whose FP64 units issue about two FMAs per clock per SM, it runs the block steps at the
   memory system's rate instead of the FP64 pipe's. Its step values carry the FP64 values to
   about 2^-48 relative, far below the level a 1e-8 residual needs (the FP32 form's floor,
   about 2^-24 G / omega^2 with G = max_i sum_j |s_ij| / m_i, drops by 2^24). */
enum kes_refine_precision { KES_REFINE_FP64 = 0, KES_REFINE_F32X2 = 1 };

/* Result of kes_krylov_solve; host memory owned by the library. */
typedef struct kes_result {
  int64_t n;             /* problem size */
  int32_t n_pairs;       /* accepted pairs: omega in [omega_min, omega_max] and rel_res <= tol */
  int32_t k_used;        /* basis size reached (summed over the intervals of kes_block_krylov_solve) */
  int32_t breakdown;     /* 1 if the Krylov space became invariant (status KES_INFO_INVARIANT_SUBSPACE) */
  int32_t n_ritz;        /* Ritz values of the last projection */
  int64_t time_steps;    /* leapfrog steps taken (per start vector) */
  double* omega2;        /* [n_pairs] accepted theta = omega^2, ascending */
  double* omega;         /* [n_pairs] sqrt(theta) */
  double* rel_res;       /* [n_pairs] relative residual */
  double* abs_res;       /* [n_pairs] ||(S - theta M) x||_2 with ||x||_M = 1 (eq. res) */
  double* vectors;       /* n x n_pairs col-major, or NULL unless want_vectors */
  double* ritz_omega2;   /* [n_ritz] every Ritz value of the last projection, ascending (with several
                            intervals: each interval's projection in turn) */
  double* ritz_rel_res;  /* [n_ritz] relative residual of the in-interval ones, NaN elsewhere */
  double solve_ms;       /* wall time of the call */
  int64_t refine_steps;  /* leapfrog steps of the refinement sweeps (per filtered block; FP64 or FP32 pairs) */
  int32_t* interval;     /* [n_pairs] the filter interval whose process found each pair (0 for one interval) */
} kes_result;

/* Counters accumulated by a context since creation or kes_reset_stats. */
typedef struct kes_stats {
  int64_t filter_calls;     /* filter applications (one per start-vector block) */
  int64_t filter_steps;     /* fused leapfrog steps launched (kernel launches of the step kernel) */
  int64_t kernel_launches;  /* every kernel this library launched (graph nodes counted one by one) */
  double filter_ms;         /* device time of the filter applications (CUDA events on the context stream) */
  double solve_other_ms;    /* device time of orthogonalisation, projection and residuals */
  int64_t bytes_per_step;   /* algorithmic HBM bytes of one fused step (see kes_step_bytes) */
  int32_t step_variant;     /* launch shape of the step kernel in use */
  int32_t step_grid;        /* its grid size (blocks of 256 threads) */
  int32_t blk_variant;      /* launch shape of the block (SpMM) step kernel, -1 for single-vector contexts */
  int32_t blk_grid;         /* its grid size */
} kes_stats;

void kes_opts_default(kes_opts* opts);
void kes_solve_opts_default(kes_solve_opts* opts);
const char* kes_strerror(int32_t status);

/*
 * kes_create -- upload S (CSR) and the lumped mass diagonal m (Sec. 2,
 * eq. def:basisMatrixEVP with Remark 2.1) and build the device
 * format (SELL-C-sigma, C = 32).
 *   n        number of dofs (rows), 1 <= n < 2^31
 *   row_ptr  host int64[n+1], row_ptr[0] = 0, non-decreasing
 *   col      host int32[nnz], column indices in [0, n), ascending inside a row
 *   val      host float64[nnz], S values (S must be symmetric PSD; not checked beyond finiteness)
 *   m_diag   host float64[n], lumped masses, all > 0 (else KES_ERR_MASS)
 *   opts     NULL for defaults
 * On success *out owns device copies; release with kes_destroy().
 */
kes_status kes_create(kes_ctx** out, int64_t n, const int64_t* row_ptr, const int32_t* col,
                      const double* val, const double* m_diag, const kes_opts* opts);
void kes_destroy(kes_ctx* ctx);
int64_t kes_size(const kes_ctx* ctx);   /* n_total: rows of all meshes */
int32_t kes_mesh_count(const kes_ctx* ctx);
kes_status kes_sync(kes_ctx* ctx);

/*
 * kes_create_batch -- several independent pencils ("meshes") in one context. They
 * are stacked block-diagonally in one SELL-C-sigma matrix, each mesh starting on a
 * slice boundary, so that every fused-step launch (and the one CUDA graph of a
 * filter application) advances all meshes at once; each mesh keeps its own tau,
 * weight tables, Krylov basis and projected problem. Arguments per mesh j < n_mesh
 * as in kes_create (host arrays: n[j], row_ptr[j], col[j], val[j], m_diag[j]).
 * Every vector passed to the other calls concatenates the meshes in this order,
 * n_total = sum_j n[j] rows per column. kes_create is the n_mesh = 1 case.
 */
kes_status kes_create_batch(kes_ctx** out, int32_t n_mesh, const int64_t* n, const int64_t* const* row_ptr,
                            const int32_t* const* col, const double* const* val, const double* const* m_diag,
                            const kes_opts* opts);

/*
 * kes_estimate_omega_max -- largest eigenfrequency of the pencil by power
 * iteration on M^{-1} S (Sec. 3.1: the stable time step is found by a power
 * iteration). v <- M^{-1} S v / ||M^{-1} S v||_2, `iters` times from the host
 * vector v0[n]; *omega_max = sqrt((v^T S v) / (v^T M v)). A power iteration
 * approaches the largest value from below; the CFL condition tau < 2/omega
 * (Sec. 2.3, after eq. scalartimestep) is why callers take tau = 0.9 * 2 / omega_max.
 * *gershgorin (may be NULL) receives the upper bound sqrt(max_i sum_j |s_ij| / m_i).
 */
kes_status kes_estimate_omega_max(kes_ctx* ctx, int32_t iters, const double* v0, double* omega_max,
                                  double* gershgorin);
/* The same power iteration for every mesh of a batch at once (each mesh normalised on
   its own rows): v0[n_total], omega_max[n_mesh], gershgorin[n_mesh] (may be NULL).
   kes_estimate_omega_max requires a single mesh (else KES_ERR_UNSUPPORTED). */
kes_status kes_estimate_omega_max_batch(kes_ctx* ctx, int32_t iters, const double* v0, double* omega_max,
                                        double* gershgorin);

/*
 * kes_set_filter -- weights alpha_n = tau * alpha(n tau), n = 0..L, of
 * eq. (weightf) sampled by the rectangle rule of eq. (disc_filtercoeff),
 * with T = L tau. L is the number of leapfrog steps (L+1 weighted samples,
 * the last at t = T). Requires 0 <= omega_min < omega_max, tau > 0, L >= 1.
 * Returns KES_ERR_UNSTABLE if tau times the last power-iteration estimate of
 * omega_max (a lower bound of it) reaches the stepper's bound, 2 (leapfrog) or
 * 2 sqrt(3) (fourth order): the CFL condition is then violated for certain.
 * With the fourth-order stepper the filter factor is sum_n alpha_n q_n(omega) with
 * that stepper's q_n (see kes_weights_response for the leapfrog's).
 * kes_set_filters sets F weight tables (intervals) that share tau and L;
 * kes_filter_apply then returns F filtered blocks from one trajectory.
 */
kes_status kes_set_filter(kes_ctx* ctx, double omega_min, double omega_max, double tau, int32_t L);
kes_status kes_set_filters(kes_ctx* ctx, int32_t F, const double* omega_min, const double* omega_max,
                           double tau, int32_t L);
/* Per-mesh filters of a batch: omega_min/omega_max[n_mesh * F] (mesh-major), tau[n_mesh];
   all meshes share L (one launch per step advances them together). kes_set_filter(s)
   give every mesh the same intervals and tau. */
kes_status kes_set_filters_batch(kes_ctx* ctx, int32_t F, const double* omega_min, const double* omega_max,
                                 const double* tau, int32_t L);
/* kes_set_weights -- any weight tables in place of eq. (weightf) (Sec. 4, "Weight
   function": the method is not tied to the indicator; e.g. a Gaussian peak).
   alpha[n_mesh][F][L+1] are the rectangle-rule weights tau * alpha(n tau) of eq.
   (disc_filtercoeff); omega_min/omega_max[n_mesh * F] is the band in which the
   solver accepts Ritz pairs; tau[n_mesh]. Same checks as kes_set_filters_batch;
   non-finite weights return KES_ERR_ARG. */
kes_status kes_set_weights(kes_ctx* ctx, int32_t F, const double* alpha, const double* omega_min,
                           const double* omega_max, const double* tau, int32_t L);

/* Host helpers, no context and no GPU needed. */
/* kes_alpha_table: alpha[0..L] = tau * alpha(n tau) of eq. (weightf), T = L tau. */
kes_status kes_alpha_table(double omega_min, double omega_max, double tau, int32_t L, double* alpha);
/* kes_filter_response: beta~(omega_i), i < k, of eq. (fullydiscfilter), the factor that
   the filter applies to an eigenvector of frequency omega (Lemma 2.3). */
kes_status kes_filter_response(double omega_min, double omega_max, double tau, int32_t L,
                               const double* omega, int64_t k, double* beta);
/* kes_weights_response: the same factor for any weight table alpha[0..L] (e.g. from
   kes_alpha_gaussian): beta~(omega_i) = sum_n alpha_n q_n(omega_i), eq. (fullydiscfilter). */
kes_status kes_weights_response(const double* alpha, double tau, int32_t L, const double* omega, int64_t k,
                                double* beta);
/* kes_alpha_gaussian: alpha[0..L] = tau * alpha(n tau) for the Gaussian pass band
   beta(omega) ~ exp(-(omega - center)^2 / (2 sigma^2)): by the inverse cosine transform
   behind eq. (filterf), alpha(t) = 2 sigma sqrt(2/pi) exp(-sigma^2 t^2 / 2) cos(center t)
   (Sec. 4, "Weight function"). Requires center >= 0, sigma > 0, tau > 0, L >= 1. */
kes_status kes_alpha_gaussian(double center, double sigma, double tau, int32_t L, double* alpha);
/* kes_alpha_triangle: the same for the triangular band beta(omega) = max(0, 1 - |omega - center| / half_width):
   alpha(t) = (2 half_width / pi) cos(center t) (sin(t half_width / 2) / (t half_width / 2))^2.
   Requires center >= 0, half_width > 0, tau > 0, L >= 1. */
kes_status kes_alpha_triangle(double center, double half_width, double tau, int32_t L, double* alpha);
/* kes_sym_eig: eigenvalues (ascending, w[k]) and orthonormal eigenvectors (V, k x k col-major,
   may be NULL) of the symmetric k x k col-major matrix A (only its lower triangle is read).
   This is the small projected problem of eq. (projevp) with B^T M B = I. */
kes_status kes_sym_eig(int32_t k, const double* A, double* w, double* V);
/* kes_launch_shapes: the number of launch shapes of the single-vector step kernel
   (kes_opts.step_variant) and of the block step kernel (kes_opts.blk_variant). */
void kes_launch_shapes(int32_t* n_step, int32_t* n_block);
/* kes_step_bytes: algorithmic HBM bytes of one fused leapfrog step of this context for b vectors
   and F intervals (every matrix entry, row pointer and per-row vector read or written once; an
   entry is its value plus a 2-byte column difference when the compact index is in use, else a
   4-byte column; the fourth-order stepper adds its stage pass and the read of the stage). The
   step kernels add the weighted terms of eq. (disc_filtercoeff) to their accumulators every third
   step and at the last (a step holds u_{n-1}, u_n, u_{n+1}), so the accumulator bytes count with
   that share of a filter application of the context's filter length L (the average step). */
int64_t kes_step_bytes(const kes_ctx* ctx, int32_t b, int32_t F);

/*
 * kes_filter_apply -- r_out = C r_in for b vectors (eq. disc_filtercoeff): L
 * leapfrog steps y_{l+1} = -tau^2 M^{-1} S y_l + 2 y_l - y_{l-1}, y_{-1} = y_0 = r
 * (eq. 2stepmethod), accumulating sum_{n=0..L} alpha_n y_n. Each step is one
 * fused kernel (SpMV, diagonal scale, three-term update, weighted accumulation).
 *   r_in   n_total x b col-major float64 (host or device per `mem`)
 *   r_out  F x b x n_total float64 (block f holds the sum with weight table f)
 *   b      1 <= b <= opts.block_b; the b vectors share one trajectory (SpMM step)
 * Device pointers: asynchronous on the context stream. Host pointers: the
 * call copies in, runs and copies out before returning.
 * KES_ERR_UNSTABLE if a non-finite value appeared in the state.
 */
kes_status kes_filter_apply(kes_ctx* ctx, const double* r_in, double* r_out, int32_t b, int32_t mem);

/*
 * kes_filter_apply_columns -- the b columns carry the trajectories of F different
 * filters (the F weight tables of kes_set_filters): column j is filtered with table
 * j / (b / F) only, so F intervals share one matrix stream. Each column's sum is the
 * one kes_filter_apply forms with that table, rounded the same way.
 *   r_in   n_total x b col-major float64 (host or device per `mem`)
 *   r_out  n_total x b col-major float64: r_out_j = C_{j / (b / F)} r_in_j
 *   b      2 <= b <= opts.block_b and a multiple of F (with F = 1, see kes_filter_apply)
 * KES_ERR_ARG if b is not a multiple of F or b < 2; otherwise as kes_filter_apply.
 */
kes_status kes_filter_apply_columns(kes_ctx* ctx, const double* r_in, double* r_out, int32_t b, int32_t mem);

/*
 * kes_krylov_solve -- Krylov space of C from r0 (Algorithm 2.5, with the
 * M-inner product and two classical Gram-Schmidt passes), Rayleigh-Ritz on it
 * (eq. projevp) and residual acceptance (eq. res).
 *   r0     start vector, length n (host or device per `mem`); it is M-normalised first
 *   sopts  NULL for defaults
 *   out    receives a kes_result (free with kes_result_free); set even on
 *          KES_INFO_INVARIANT_SUBSPACE.
 * Requires a single mesh and a single filter interval (kes_set_filter).
 */
kes_status kes_krylov_solve(kes_ctx* ctx, const double* r0, int32_t mem, const kes_solve_opts* sopts,
                            kes_result** out);

/*
 * kes_block_krylov_solve -- the block version of the Krylov space (Sec. 4: start
 * from b M-orthonormalised random vectors and orthonormalise every filtered block),
 * for every mesh of the context at once. Each block step filters the b newest basis
 * vectors of every mesh in one SpMM trajectory, then orthogonalises each filtered
 * vector (two classical passes, M-inner product) into its mesh's basis; dependent
 * vectors are dropped, and a mesh whose whole block is dependent stops (invariant
 * subspace). The projected problem and the residual acceptance are those of
 * kes_krylov_solve, per mesh. A block of b vectors resolves eigenvalues of
 * multiplicity up to b.
 *   R0     n_total x b col-major start vectors (host or device per `mem`)
 *   b      1 <= b <= opts.block_b
 *   sopts  kmax counts basis vectors per mesh and interval (kmax >= b / F)
 *   out    array of kes_mesh_count(ctx) result pointers, one per mesh (free each with
 *          kes_result_free); set on KES_OK and KES_INFO_INVARIANT_SUBSPACE
 * Several intervals (kes_set_filters with F > 1) run as F independent block solvers
 * that share the matrix stream: b must be a multiple of F, and interval f owns the
 * g = b / F columns f g .. f g + g - 1 of the start block and of every block step,
 * filtered with its own weights (kes_filter_apply_columns). Each interval keeps its
 * own basis (kmax vectors), projection and acceptance, exactly as a separate call with
 * its g start vectors would; the accepted pairs of a mesh are merged in ascending
 * omega and kes_result.interval names the interval of each (a pair that lies in two
 * overlapping intervals can be reported by both). n_wanted counts a mesh's pairs over
 * all its intervals. The refinement sweeps filter each interval's Ritz vectors with
 * that interval's weights.
 * KES_ERR_ARG if b is not a multiple of F or kmax < b / F.
 */
kes_status kes_block_krylov_solve(kes_ctx* ctx, const double* R0, int32_t b, int32_t mem,
                                  const kes_solve_opts* sopts, kes_result** out);

/*
 * kes_subspace_solve -- the fixed-dimension alternative of Sec. 4 (a FEAST-like
 * iteration with the time-domain filter): from the p columns of X0, each of
 * sopts->refine_sweeps sweeps filters every vector (X <- C X, in the context's
 * precision, sopts->refine_L steps if set), M-orthonormalises the results (dependent
 * ones dropped), solves the projected problem (eq. projevp) and feeds all of its Ritz
 * vectors to the next sweep, so memory stays at p basis vectors per mesh. The pairs of
 * the last sweep in the interval with rel_res <= tol are returned. The iteration
 * converges to the p eigenvectors with the largest |beta~|: choose p above the number
 * of eigenvalues in the interval.
 *   X0     n_total x p col-major (host or device per `mem`); every mesh starts from its rows
 *   sopts  refine_sweeps >= 1 (the sweeps), kmax >= p, tol; check_every and n_wanted unused
 *   out    array of kes_mesh_count(ctx) result pointers (time_steps = 0, refine_steps = the
 *          leapfrog steps of the sweeps per filtered block)
 * Requires a single interval per mesh (KES_ERR_UNSUPPORTED otherwise).
 */
kes_status kes_subspace_solve(kes_ctx* ctx, const double* X0, int32_t p, int32_t mem, const kes_solve_opts* sopts,
                              kes_result** out);
void kes_result_free(kes_result* res);

kes_status kes_get_stats(kes_ctx* ctx, kes_stats* stats); /* synchronises the stream */
kes_status kes_reset_stats(kes_ctx* ctx);

/*
 * kes_filter_apply_noalloc -- r_out = C r_in for one start vector in FP64, like
 * kes_filter_apply, without allocating anything. The paper has no counterpart:
 * this entry point is for callers that cannot call cudaMalloc at all, such as a
 * program that reserves every byte of device memory it may use when it starts and
 * forbids later allocation (a long-running service with a fixed memory budget, a
 * plugin whose host owns the device heap), so that nothing can fail or fragment
 * mid-run. kes_create allocates the context's state, so those callers use this
 * function: they own every input and the output, and the two leapfrog state
 * vectors live in a fixed array inside the library, 2 * KES_NOALLOC_MAX_N doubles
 * (16 MiB), which every GPU where the library's module is loaded holds until the
 * process exits.
 *   n        rows, 1 <= n <= KES_NOALLOC_MAX_N; a larger n returns KES_ERR_ARG and launches nothing
 *   row_ptr  device int64[n+1]; col device int32[nnz]; val device float64[nnz]: CSR of S
 *   tau2m    device float64[n], tau^2 / m_i
 *   alpha    device float64[L+1], the weights kes_alpha_table returns (L >= 1 steps)
 *   r_in     device float64[n]; r_out device float64[n] receives the filtered vector
 *   stream   cudaStream_t (NULL: the legacy default stream); the call only enqueues the work
 * Preconditions that are NOT checked (the arrays stay on the device, unlike kes_create's):
 * row_ptr[0] = 0, row_ptr non-decreasing, row_ptr[n] = nnz; every col entry in [0, n);
 * every array of the stated length and on the current device. A violation is an
 * out-of-bounds device access, not an error status.
 * Set-up: the first call on a device loads the library's module there (CUDA loads
 * modules lazily by default), which takes the 16 MiB array and the module's code from
 * device memory, and looks up the array's address (once per device, with that device
 * current). A caller that reserves all of its device memory must make one call before
 * it does (or run with CUDA_MODULE_LOADING=EAGER); make that first call before any
 * stream capture as well. Every call shares the array, which keeps the last call's
 * contents (each call writes every entry before reading it, so nothing needs
 * clearing); calls whose GPU work overlaps race on it. A CFL violation is not detected
 * here: it shows as huge or non-finite values in r_out. Calls no cudaMalloc, cudaFree
 * or other allocating routine.
 */
#define KES_NOALLOC_MAX_N 1048576
kes_status kes_filter_apply_noalloc(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                                    const double* tau2m, const double* alpha, int32_t L, const double* r_in,
                                    double* r_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KES_H */
