// Fused leapfrog step kernels on SELL-C-sigma (C = 32), sm_103a.
//
// One step of the filter application (Sec. 2.3, eq. 2stepmethod and
// eq. disc_filtercoeff; Algorithm 2.5, time loop):
//   u_{n+1} = 2 u_n - u_{n-1} - tau^2 M^{-1} S u_n = (2 u_n - u_{n-1}) + A u_n
//   acc_f  += alpha_f[n+1] * u_{n+1}
// with A = -tau^2 M^{-1} S stored once per kes_set_filter (the diagonal scale is
// folded into the values), fused into one pass: a warp owns one 32-row slice
// (lane = row); the slice's values and column indices stream from HBM in
// 256-byte (FP64) / 128-byte (FP32) coalesced warp loads marked evict-first, u_n
// is gathered through the read-only path (it stays L2-resident across the step),
// and each row is one FMA chain seeded with 2 u_n - u_{n-1}. The weighted terms
// alpha_f[m] u_m reach the accumulators in every third step (and the last), which
// adds the pending ones of u_{n-1}, u_n, u_{n+1} from registers in index order.
// No tensor cores: the step is a sparse gather, not a dense contraction.
#include <cuda_runtime.h>

#include "kes_internal.h"

namespace kes {

thread_local int64_t g_launches = 0;

namespace {

__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_stream(const int16_t* p) { return __ldcs(reinterpret_cast<const short*>(p)); }

// init + sum_k val[32k] * x[col_k] over the w entries of one lane's row, one FMA
// chain in entry order (every step kernel forms it the same way, so all launch
// shapes round identically). Loads are issued BATCH entries at a time. The column is
// base + c[32k]: absolute int32 columns with base 0, or 16-bit column - row
// differences with base = row (the compact index SellDev::dcol).
template <typename T, int BATCH, typename I>
__device__ __forceinline__ T row_dot(T acc, const T* __restrict__ v, const I* __restrict__ c, int base, int w,
                                     const T* __restrict__ x) {
  int k = 0;
  for (; k + BATCH <= w; k += BATCH) {
    int32_t cc[BATCH];
    T vv[BATCH], xx[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; ++j) cc[j] = base + ld_stream(c + (k + j) * kSliceC);
#pragma unroll
    for (int j = 0; j < BATCH; ++j) vv[j] = ld_stream(v + (k + j) * kSliceC);
#pragma unroll
    for (int j = 0; j < BATCH; ++j) xx[j] = __ldg(x + cc[j]);
#pragma unroll
    for (int j = 0; j < BATCH; ++j) acc = fma(vv[j], xx[j], acc);
  }
  if (k < w) {
    int32_t cc[BATCH];
    T vv[BATCH], xx[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; ++j)
      if (k + j < w) cc[j] = base + ld_stream(c + (k + j) * kSliceC);
#pragma unroll
    for (int j = 0; j < BATCH; ++j)
      if (k + j < w) vv[j] = ld_stream(v + (k + j) * kSliceC);
#pragma unroll
    for (int j = 0; j < BATCH; ++j)
      if (k + j < w) xx[j] = __ldg(x + cc[j]);
#pragma unroll
    for (int j = 0; j < BATCH; ++j)
      if (k + j < w) acc = fma(vv[j], xx[j], acc);
  }
  return acc;
}

// g is the vector the row sums gather from: u_n itself for the leapfrog, the stage
// v = u_n + A u_n / 12 for the fourth-order scheme; x = u_n seeds the row (2 u_n - u_{n-1}).
// The same sum over the pair layout: pair p of the lane holds entries 2p and 2p+1 (one
// float2 / double2 of values, one 32-bit word of two 16-bit column differences, low half first),
// NP pairs' loads issued together; the chain is still in entry order. w is the row's
// number of entries: for odd w the last pair's second entry is padding. Its pair is loaded
// with its batch (no extra round trip) but the padding is neither gathered nor summed.
template <typename T> struct Pair2;
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<double> { using type = double2; };

template <typename T, int NP>
__device__ __forceinline__ T row_dot_pairs(T acc, const typename Pair2<T>::type* __restrict__ v,
                                           const int32_t* __restrict__ c, int row, int w, const T* __restrict__ x) {
  using T2 = typename Pair2<T>::type;
  const int wp = w >> 1;          // full pairs
  const int wpp = (w + 1) >> 1;   // stored pairs
  int k = 0;
  for (; k + NP <= wpp; k += NP) {
    int32_t cc[NP];
    T2 vv[NP];
    T xa[NP], xb[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) cc[j] = __ldcs(c + (k + j) * kSliceC);
#pragma unroll
    for (int j = 0; j < NP; ++j) vv[j] = __ldcs(v + (k + j) * kSliceC);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      xa[j] = __ldg(x + row + static_cast<int16_t>(cc[j] & 0xffff));
      xb[j] = k + j < wp ? __ldg(x + row + (cc[j] >> 16)) : T(0);
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      acc = fma(vv[j].x, xa[j], acc);
      if (k + j < wp) acc = fma(vv[j].y, xb[j], acc);
    }
  }
  for (; k < wpp; ++k) {
    const int32_t c0 = __ldcs(c + k * kSliceC);
    const T2 v0 = __ldcs(v + k * kSliceC);
    const T a = __ldg(x + row + static_cast<int16_t>(c0 & 0xffff));
    const T b = k < wp ? __ldg(x + row + (c0 >> 16)) : T(0);
    acc = fma(v0.x, a, acc);
    if (k < wp) acc = fma(v0.y, b, acc);
  }
  return acc;
}

// IDX: how the row sums read columns: 0 the int32 columns, 1 the compact 16-bit column -
// row differences (A.dcol), 2 the pair layout (A.val64p, A.dcolp); one form per
// instantiation keeps a single loop in the kernel. With A.fold2 the values hold A + 2I (the
// 2 u_n of eq. 2stepmethod folded into the diagonal; only for the leapfrog, where g = x) and
// the row seeds with -u_{n-1} alone: one FP64 operation less per row. The pair values are
// built only in that form, so IDX 2 implies it.
//
// Accumulation: with ACC the step adds the last nterm (1-3) of alpha_{n-1} u_{n-1},
// alpha_n u_n, alpha_{n+1} u_{n+1} (all three are in registers) in that order, the first of
// them as a product when init (the accumulator's first terms); without ACC it leaves the
// accumulators alone. The host runs the accumulation every third step and at the last, so
// every term is added once, in index order, with the operations of adding one per step.
template <bool FIRST, bool LAST, bool ACC, int BATCH, int MINB, int IDX>
__global__ void __launch_bounds__(256, MINB) k_step_f64(SellDev A, const double* __restrict__ x,
                                                  const double* __restrict__ g, const double* prev,
                                                  double* out, double* acc, int64_t acc_stride, int F,
                                                  const double* __restrict__ alpha, int Lp1, int step,
                                                  int nterm, int init, int* flag) {
  static_assert(ACC || !LAST, "the last step completes the sums");
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < A.n_slices;
       s += nwarps) {
    const int64_t beg = A.slice_ptr[s];
    const int w = static_cast<int>((A.slice_ptr[s + 1] - beg) >> 5);
    const int64_t row = s * kSliceC + lane;
    const int64_t mesh = A.slice_mesh ? A.slice_mesh[s] : 0;
    const double xi = x[row];
    const double pi = FIRST ? xi : prev[row];
    const double seed = (IDX == 2 || A.fold2) ? -pi : 2.0 * xi - pi;
    double un;
    if constexpr (IDX == 2) {
      const int64_t b2 = A.slice_ptr2[s];
      un = row_dot_pairs<double, (BATCH >= 2 ? BATCH / 2 : 1)>(
          seed, reinterpret_cast<const double2*>(A.val64p + b2) + lane,
          reinterpret_cast<const int32_t*>(A.dcolp + b2) + lane, static_cast<int>(row), w, g);
    } else if constexpr (IDX == 1) {
      un = row_dot<double, BATCH>(seed, A.val64 + beg + lane, A.dcol + beg + lane, static_cast<int>(row), w, g);
    } else {
      un = row_dot<double, BATCH>(seed, A.val64 + beg + lane, A.col + beg + lane, 0, w, g);
    }
    if (!LAST) out[row] = un;
    if constexpr (ACC) {
      bool bad = false;
      const int t0 = 3 - nterm;  // term t is alpha_m u_m, m = step - 1 + t
      for (int f = 0; f < F; ++f) {
        const int64_t ab = (mesh * F + f) * Lp1 + step - 1;
        double* a = acc + f * acc_stride + row;
        double na = init ? 0.0 : *a;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          if (t < t0) continue;
          const double u = t == 0 ? pi : (t == 1 ? xi : un);
          const double h = alpha[ab + t];
          na = (init && t == t0) ? h * u : fma(h, u, na);
        }
        *a = na;
        if (LAST) bad |= !isfinite(na);
      }
      if (LAST && bad) atomicOr(flag, 1);
    }
  }
}

// error-free sum: s + t = a + b exactly (Knuth's two-sum), round-to-nearest ops only
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  t = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// IDX: 0 int32 columns, 1 the compact 16-bit differences, 2 the pair layout.
// ACC and nterm as in k_step_f64 (the accumulators start from k_init_f32).
template <bool FIRST, bool LAST, bool ACC, int BATCH, int MINB, int IDX>
__global__ void __launch_bounds__(256, MINB) k_step_f32(SellDev A, const float* __restrict__ x,
                                                  const float* __restrict__ g, const float* prev,
                                                  float* out, float* acc_s, float* acc_c, double* acc64,
                                                  int64_t acc_stride, int F, const float* __restrict__ ahi,
                                                  const float* __restrict__ alo, int Lp1, int step,
                                                  int nterm, int* flag) {
  static_assert(ACC || !LAST, "the last step completes the sums");
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < A.n_slices;
       s += nwarps) {
    const int64_t beg = A.slice_ptr[s];
    const int w = static_cast<int>((A.slice_ptr[s + 1] - beg) >> 5);
    const int64_t row = s * kSliceC + lane;
    const int64_t mesh = A.slice_mesh ? A.slice_mesh[s] : 0;
    const float xi = x[row];
    const float pi = FIRST ? xi : prev[row];
    const float seed = __fsub_rn(__fmul_rn(2.0f, xi), pi);
    float un;
    if constexpr (IDX == 2) {
      const int64_t b2 = A.slice_ptr2[s];
      un = row_dot_pairs<float, (BATCH >= 2 ? BATCH / 2 : 1)>(
          seed, reinterpret_cast<const float2*>(A.val32p + b2) + lane,
          reinterpret_cast<const int32_t*>(A.dcolp + b2) + lane, static_cast<int>(row), w, g);
    } else if constexpr (IDX == 1) {
      un = row_dot<float, BATCH>(seed, A.val32 + beg + lane, A.dcol + beg + lane, static_cast<int>(row), w, g);
    } else {
      un = row_dot<float, BATCH>(seed, A.val32 + beg + lane, A.col + beg + lane, 0, w, g);
    }
    if (!LAST) out[row] = un;
    if constexpr (ACC) {
      bool bad = false;
      const int t0 = 3 - nterm;  // term t is alpha_m u_m, m = step - 1 + t
      for (int f = 0; f < F; ++f) {
        const int64_t ab = (mesh * F + f) * Lp1 + step - 1;
        const int64_t at = f * acc_stride + row;
        float sa = acc_s[at], ca = acc_c[at];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          if (t < t0) continue;
          const float u = t == 0 ? pi : (t == 1 ? xi : un);
          const float a_hi = ahi[ab + t], a_lo = alo[ab + t];
          // alpha * u = p + pe, p = fl(a_hi * u), pe = (a_hi * u - p) + a_lo * u
          const float p = __fmul_rn(a_hi, u);
          const float pe = fmaf(a_lo, u, fmaf(a_hi, u, -p));
          float sn, e;
          two_sum(sa, p, sn, e);
          ca = __fadd_rn(ca, __fadd_rn(e, pe));
          sa = sn;
        }
        if (LAST) {
          const double v = static_cast<double>(sa) + static_cast<double>(ca);
          acc64[at] = v;
          bad |= !isfinite(v);
        } else {
          acc_s[at] = sa;
          acc_c[at] = ca;
        }
      }
      if (LAST && bad) atomicOr(flag, 1);
    }
  }
}

// FP32 start for nb columns (row-major, nb values per row): x32 = (float) r64 and the
// compensated accumulator of weight table f set to alpha_f[0] r, split as s + c (cpt > 0:
// one accumulator per column, with table min(column / cpt, F - 1)).
__global__ void k_init_f32(int64_t count, int nb, const double* __restrict__ r, float* __restrict__ x32,
                           float* __restrict__ acc_s, float* __restrict__ acc_c, int64_t acc_stride, int F,
                           const double* __restrict__ alpha, int Lp1, const int32_t* __restrict__ slice_mesh,
                           int cpt) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double ri = r[i];
    const int64_t mesh = slice_mesh ? slice_mesh[(i / nb) / kSliceC] : 0;
    x32[i] = static_cast<float>(ri);
    const int nacc = cpt ? 1 : F;
    for (int f = 0; f < nacc; ++f) {
      const int table = cpt ? min(static_cast<int>(i % nb) / cpt, F - 1) : f;
      const double t = alpha[(mesh * F + table) * Lp1] * ri;
      const float s = static_cast<float>(t);
      acc_s[f * acc_stride + i] = s;
      acc_c[f * acc_stride + i] = static_cast<float>(t - static_cast<double>(s));
    }
  }
}

__global__ void __launch_bounds__(256) k_spmv_f64(SellDev A, const double* __restrict__ x,
                                                  const double* __restrict__ dscale, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < A.n_slices;
       s += nwarps) {
    const int64_t beg = A.slice_ptr[s];
    const int w = static_cast<int>((A.slice_ptr[s + 1] - beg) >> 5);
    const double sum = row_dot<double, 8>(0.0, A.val64 + beg + lane, A.col + beg + lane, 0, w, x);
    const int64_t row = s * kSliceC + lane;
    y[row] = dscale ? sum * dscale[row] : sum;
  }
}

// A = -tau^2 M^{-1} S in the SELL layout: out[e] = -tau2m[row(e)] * val64[e]
// (out64p / out32p: the same values in the pair layout of A.slice_ptr2; their padding
// entries keep the zeros they were allocated with. fold2: out64 and out64p hold A + 2I, 2
// added to the first entry of each row at its own column, which the context has checked
// exists: a stored diagonal, or SELL padding, which points at its own row.)
__global__ void k_scale_values(SellDev A, const double* __restrict__ tau2m, double* __restrict__ out64,
                               float* __restrict__ out32, double* __restrict__ out64p,
                               float* __restrict__ out32p, int fold2) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < A.n_slices;
       s += nwarps) {
    const int64_t beg = A.slice_ptr[s], end = A.slice_ptr[s + 1];
    const double t = -tau2m[s * kSliceC + lane];
    const int64_t row = s * kSliceC + lane;
    bool diag_done = false;
    int k = 0;
    for (int64_t e = beg + lane; e < end; e += kSliceC, ++k) {
      const double a = t * A.val64[e];
      const bool fold = fold2 && !diag_done && A.col[e] == row;
      diag_done |= fold;
      if (out64) out64[e] = fold ? a + 2.0 : a;
      if (out32) out32[e] = static_cast<float>(a);
      const int64_t p2 = A.slice_ptr2 ? A.slice_ptr2[s] + 64 * (k >> 1) + 2 * lane + (k & 1) : 0;
      if (out64p) out64p[p2] = fold ? a + 2.0 : a;
      if (out32p) out32p[p2] = static_cast<float>(a);
    }
  }
}

__global__ void k_check_finite(const double* __restrict__ v, int64_t n, int* flag) {
  bool bad = false;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    bad |= !isfinite(v[i]);
  if (bad) atomicOr(flag, 1);
}

int grid_for(const LaunchCfg& cfg, int64_t n_slices) {
  const int64_t need = (n_slices + (cfg.block_step / 32) - 1) / (cfg.block_step / 32);
  return static_cast<int>(need < cfg.grid_step ? need : cfg.grid_step);
}

// Launch shapes of the step kernels: (load batch, minimum resident blocks of 256
// threads per SM, which caps the registers). Every variant computes the same sums.
// (An L2 prefetch of each warp's next slice was measured as well: 8-50% slower on the
// 128^3 cube in every shape, so it is not offered.)
#define KES_STEP_VARIANTS(X) \
  X(0, 8, 1) X(1, 8, 3) X(2, 8, 4) X(3, 4, 4) X(4, 4, 5) X(5, 4, 6) X(6, 2, 6) X(7, 2, 8)

// first / last / accumulating forms of one instantiation (the first step accumulates only
// when it is the last as well: it holds at most two of the pending terms)
#define KES_STEP_FORMS(KERNEL, I, ARGS)                                                                   \
  if (last) {                                                                                             \
    if (first) KERNEL<true, true, true, BATCH, MINB, I><<<grid, block, 0, st>>>(ARGS);                    \
    else KERNEL<false, true, true, BATCH, MINB, I><<<grid, block, 0, st>>>(ARGS);                         \
  } else if (first) {                                                                                     \
    KERNEL<true, false, false, BATCH, MINB, I><<<grid, block, 0, st>>>(ARGS);                             \
  } else if (nterm) {                                                                                     \
    KERNEL<false, false, true, BATCH, MINB, I><<<grid, block, 0, st>>>(ARGS);                             \
  } else {                                                                                                \
    KERNEL<false, false, false, BATCH, MINB, I><<<grid, block, 0, st>>>(ARGS);                            \
  }

template <int BATCH, int MINB>
void step_f64_impl(int grid, int block, cudaStream_t st, bool first, bool last, const SellDev& A, const double* x,
                   const double* g, const double* prev, double* out, double* acc, int64_t acc_stride, int F, const double* alpha,
                   int Lp1, int step, int nterm, int init, int* flag) {
#define KES_F64_ARGS A, x, g, prev, out, acc, acc_stride, F, alpha, Lp1, step, nterm, init, flag
#define KES_F64_LAUNCH(I) KES_STEP_FORMS(k_step_f64, I, KES_F64_ARGS)
  if (A.val64p && A.fold2) {  // the pair form seeds with -u_{n-1}: the values must hold A + 2I
    KES_F64_LAUNCH(2)
  } else if (A.dcol) {
    KES_F64_LAUNCH(1)
  } else {
    KES_F64_LAUNCH(0)
  }
#undef KES_F64_LAUNCH
#undef KES_F64_ARGS
}

template <int BATCH, int MINB>
void step_f32_impl(int grid, int block, cudaStream_t st, bool first, bool last, const SellDev& A, const float* x,
                   const float* g, const float* prev, float* out, float* acc_s, float* acc_c, double* acc64, int64_t acc_stride,
                   int F, const float* ahi, const float* alo, int Lp1, int step, int nterm, int* flag) {
#define KES_F32_ARGS A, x, g, prev, out, acc_s, acc_c, acc64, acc_stride, F, ahi, alo, Lp1, step, nterm, flag
#define KES_F32_LAUNCH(I) KES_STEP_FORMS(k_step_f32, I, KES_F32_ARGS)
  if (A.val32p) {
    KES_F32_LAUNCH(2)
  } else if (A.dcol) {
    KES_F32_LAUNCH(1)
  } else {
    KES_F32_LAUNCH(0)
  }
#undef KES_F32_LAUNCH
#undef KES_F32_ARGS
}
#undef KES_STEP_FORMS

}  // namespace

int step_variant_count() {
  int n = 0;
#define X(ID, B, M) ++n;
  KES_STEP_VARIANTS(X)
#undef X
  return n;
}

int step_blocks_per_sm(bool fp32, int variant, int block) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (variant) {
#define X(ID, B, M)                                                                                      \
  case ID:                                                                                               \
    e = fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_f32<false, false, true, B, M, 2>, block, 0) \
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_f64<false, false, true, B, M, 2>, block, 0); \
    break;
    KES_STEP_VARIANTS(X)
#undef X
    default: break;
  }
  return (e == cudaSuccess && nb > 0) ? nb : 2;
}

void launch_step_f64(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, bool first, const double* x,
                     const double* g, const double* prev, double* out, double* acc, int64_t acc_stride, int F,
                     const double* alpha, int L, int step, bool last, int nterm, bool init, int* flag) {
  const int grid = grid_for(cfg, A.n_slices);
  switch (cfg.variant) {
#define X(ID, B, M)                                                                                        \
  case ID:                                                                                                 \
    step_f64_impl<B, M>(grid, cfg.block_step, st, first, last, A, x, g, prev, out, acc, acc_stride, F,     \
                        alpha, L + 1, step, nterm, init ? 1 : 0, flag);                                    \
    break;
    KES_STEP_VARIANTS(X)
#undef X
    default: break;
  }
  ++g_launches;
}

void launch_step_f32(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, bool first, bool last, const float* x,
                     const float* g, const float* prev, float* out, float* acc_s, float* acc_c, double* acc64,
                     int64_t acc_stride, int F, const float* alpha_hi, const float* alpha_lo, int L, int step,
                     int nterm, int* flag) {
  const int grid = grid_for(cfg, A.n_slices);
  switch (cfg.variant) {
#define X(ID, B, M)                                                                                        \
  case ID:                                                                                                 \
    step_f32_impl<B, M>(grid, cfg.block_step, st, first, last, A, x, g, prev, out, acc_s, acc_c, acc64,     \
                        acc_stride, F, alpha_hi, alpha_lo, L + 1, step, nterm, flag);                      \
    break;
    KES_STEP_VARIANTS(X)
#undef X
    default: break;
  }
  ++g_launches;
}

void launch_init_f32(cudaStream_t st, const SellDev& A, int nb, const double* r64, float* x32, float* acc_s,
                     float* acc_c, int64_t acc_stride, int F, const double* alpha64, int L, int cpt) {
  const int64_t count = A.n_pad * nb;
  const int64_t blocks = (count + 255) / 256;
  k_init_f32<<<static_cast<int>(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(
      count, nb, r64, x32, acc_s, acc_c, acc_stride, F, alpha64, L + 1, A.slice_mesh, cpt);
  ++g_launches;
}

void launch_spmv_f64(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, const double* x,
                     const double* dscale, double* y) {
  k_spmv_f64<<<grid_for(cfg, A.n_slices), cfg.block_step, 0, st>>>(A, x, dscale, y);
  ++g_launches;
}

void launch_scale_values(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, const double* tau2m,
                         double* out64, float* out32, double* out64p, float* out32p, bool fold2) {
  k_scale_values<<<grid_for(cfg, A.n_slices), cfg.block_step, 0, st>>>(A, tau2m, out64, out32, out64p, out32p,
                                                                        fold2 ? 1 : 0);
  ++g_launches;
}

void launch_check_finite(cudaStream_t st, const double* v, int64_t n, int* flag) {
  const int64_t blocks = (n + 255) / 256;
  k_check_finite<<<static_cast<int>(blocks < 2048 ? blocks : 2048), 256, 0, st>>>(v, n, flag);
  ++g_launches;
}

}  // namespace kes
