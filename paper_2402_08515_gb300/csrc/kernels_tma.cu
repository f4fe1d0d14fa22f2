// Fused leapfrog step with bulk-asynchronous (TMA) staging of the matrix, sm_103a.
//
// Same arithmetic as k_step_f64 / k_step_f32 (Sec. 2.3, eq. 2stepmethod and
// eq. disc_filtercoeff), different data movement: a CTA owns a contiguous range of
// SELL slices; one producer thread streams consecutive chunks of G slices (their
// values and column indices are two contiguous byte ranges) into a ring of S
// shared-memory stages with cp.async.bulk, completing on an mbarrier per stage;
// G consumer warps take one slice each from the stage, gather u_n from global
// memory (L2-resident) and update their 32 rows, then release the stage. The ring
// keeps S chunks of the matrix in flight per CTA independently of the consumers'
// registers, which is what the latency-bound register-staged kernel lacks.
//
// Every wait is bounded: a thread that waits more than ~2^31 cycles sets bit 1 of
// the error flag (reported as KES_ERR_TIMEOUT) and leaves its loop; before the CTA
// exits, the producer waits (again bounded) until every copy it issued has landed.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "kes_internal.h"

namespace kes {
namespace {

constexpr long long kWaitCycles = 1LL << 31;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of parity `parity` to complete; false on timeout or, when
// `give_up_on_flag`, as soon as another thread has reported a timeout (bit 1 of *flag).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* flag, bool give_up_on_flag = true) {
  const long long t0 = clock64();
  for (int it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255) {
      if (give_up_on_flag && (*reinterpret_cast<volatile int*>(flag) & 2)) return false;
      if (clock64() - t0 > kWaitCycles) {
        atomicOr(flag, 2);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  t = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

template <typename T, bool FIRST, bool LAST>
__global__ void k_step_tma(SellDev A, int G, int S, int wmax, const T* __restrict__ x, const T* prev, T* out,
                           T* acc_s, T* acc_c, double* acc64,
                           int64_t acc_stride, int F, const T* __restrict__ ahi, const T* __restrict__ alo,
                           int Lp1, int step, int* flag) {
  constexpr bool kF32 = std::is_same<T, float>::value;
  extern __shared__ __align__(128) unsigned char smem[];
  const int64_t stage_entries = static_cast<int64_t>(G) * kSliceC * wmax;
  T* sval = reinterpret_cast<T*>(smem);
  int32_t* scol = reinterpret_cast<int32_t*>(smem + S * stage_entries * sizeof(T));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * stage_entries * (sizeof(T) + sizeof(int32_t)));
  // bars[0..S): full (producer arrives with the byte count), bars[S..2S): empty (G consumers)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* gval;
  if constexpr (kF32) gval = A.val32;
  else gval = A.val64;

  // this CTA's slices and chunks
  const int64_t per = (A.n_slices + gridDim.x - 1) / gridDim.x;
  const int64_t s_begin = blockIdx.x * per;
  const int64_t s_end = min(A.n_slices, s_begin + per);
  const int64_t nchunks = s_end > s_begin ? (s_end - s_begin + G - 1) / G : 0;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_addr(&bars[i]), 1);
      mbar_init(smem_addr(&bars[S + i]), G);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == 0) {
    // ---------------- producer: one thread issues the bulk copies
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t c = 0; c < nchunks; ++c) {
        const int st = static_cast<int>(c % S);
        const uint32_t round = static_cast<uint32_t>(c / S);
        if (!mbar_wait(smem_addr(&bars[S + st]), (round & 1) ^ 1, flag)) break;
        const int64_t s0 = s_begin + c * G;
        const int64_t s1 = min(s_end, s0 + G);
        const int64_t e0 = A.slice_ptr[s0], e1 = A.slice_ptr[s1];
        const uint32_t nv = static_cast<uint32_t>((e1 - e0) * sizeof(T));
        const uint32_t nc = static_cast<uint32_t>((e1 - e0) * sizeof(int32_t));
        const uint32_t full = smem_addr(&bars[st]);
        mbar_arrive_expect_tx(full, nv + nc);
        if (nv > 0) {
          bulk_g2s(smem_addr(sval + st * stage_entries), gval + e0, nv, full);
          bulk_g2s(smem_addr(scol + st * stage_entries), A.col + e0, nc, full);
        }
        issued = c + 1;
      }
      // drain: every issued copy has landed before the CTA may exit
      for (int64_t c = issued > S ? issued - S : 0; c < issued; ++c)
        mbar_wait(smem_addr(&bars[c % S]), static_cast<uint32_t>(c / S) & 1, flag, false);
    }
  } else {
    // ---------------- consumers: warp g takes slice g of every chunk
    const int g = warp - 1;
    for (int64_t c = 0; c < nchunks; ++c) {
      const int st = static_cast<int>(c % S);
      const uint32_t round = static_cast<uint32_t>(c / S);
      if (!mbar_wait(smem_addr(&bars[st]), round & 1, flag)) break;
      const int64_t s0 = s_begin + c * G;
      const int64_t s = s0 + g;
      if (s < s_end) {
        const int64_t base = A.slice_ptr[s0];
        const int64_t beg = A.slice_ptr[s];
        const int w = static_cast<int>((A.slice_ptr[s + 1] - beg) >> 5);
        const T* v = sval + st * stage_entries + (beg - base) + lane;
        const int32_t* cl = scol + st * stage_entries + (beg - base) + lane;
        const int64_t row = s * kSliceC + lane;
        const int64_t mesh = A.slice_mesh ? A.slice_mesh[s] : 0;
        const T xi = x[row];
        const T pi = FIRST ? xi : prev[row];
        // u_{n+1} = (2 u_n - u_{n-1}) + A u_n, one FMA chain in entry order
        T un;
        if constexpr (kF32) un = __fsub_rn(__fmul_rn(2.0f, xi), pi);
        else un = A.fold2 ? -pi : 2.0 * xi - pi;  // A.fold2: 2 x is in the diagonal
        int k = 0;
        for (; k + 2 <= w; k += 2) {
          const int32_t c0 = cl[k * kSliceC], c1 = cl[(k + 1) * kSliceC];
          const T x0 = __ldg(x + c0), x1 = __ldg(x + c1);
          un = fma(v[(k + 1) * kSliceC], x1, fma(v[k * kSliceC], x0, un));
        }
        if (k < w) un = fma(v[k * kSliceC], __ldg(x + cl[k * kSliceC]), un);
        if (!LAST) out[row] = un;
        bool bad = false;
        for (int f = 0; f < F; ++f) {
          const int64_t ai = (mesh * F + f) * Lp1;
          const int64_t at = f * acc_stride + row;
          if constexpr (kF32) {
            const float a_hi = ahi[ai + step + 1], a_lo = alo[ai + step + 1];
            const float p = __fmul_rn(a_hi, un);
            const float pe = fmaf(a_lo, un, fmaf(a_hi, un, -p));
            float sn, e;
            two_sum(acc_s[at], p, sn, e);
            const float cn = __fadd_rn(acc_c[at], __fadd_rn(e, pe));
            if (LAST) {
              const double val = static_cast<double>(sn) + static_cast<double>(cn);
              acc64[at] = val;
              bad |= !isfinite(val);
            } else {
              acc_s[at] = sn;
              acc_c[at] = cn;
            }
          } else {
            const double na = fma(ahi[ai + step + 1], un, FIRST ? ahi[ai] * xi : acc_s[at]);
            acc_s[at] = na;
            if (LAST) bad |= !isfinite(na);
          }
        }
        if (LAST && bad) atomicOr(flag, 1);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&bars[S + st]));
    }
  }
}

template <typename T>
size_t tma_smem(int G, int S, int wmax) {
  return static_cast<size_t>(S) * G * kSliceC * wmax * (sizeof(T) + sizeof(int32_t)) + 2 * S * sizeof(uint64_t);
}

template <typename T, bool FIRST, bool LAST>
void tma_launch_one(const TmaShape& sh, int n_sm, cudaStream_t st, const SellDev& A, const T* x, const T* prev,
                    T* out, T* acc_s, T* acc_c, double* acc64, int64_t acc_stride, int F, const T* ahi, const T* alo,
                    int Lp1, int step, int* flag) {
  const size_t smem = tma_smem<T>(sh.G, sh.S, sh.wmax);
  k_step_tma<T, FIRST, LAST><<<n_sm * sh.ctas_per_sm, (sh.G + 1) * 32, smem, st>>>(
      A, sh.G, sh.S, sh.wmax, x, prev, out, acc_s, acc_c, acc64, acc_stride, F, ahi, alo, Lp1, step, flag);
}

template <typename T>
void tma_dispatch(const TmaShape& sh, int n_sm, cudaStream_t st, bool first, bool last, const SellDev& A, const T* x,
                  const T* prev, T* out, T* acc_s, T* acc_c, double* acc64, int64_t acc_stride, int F, const T* ahi,
                  const T* alo, int Lp1, int step, int* flag) {
#define KES_TMA_ARGS sh, n_sm, st, A, x, prev, out, acc_s, acc_c, acc64, acc_stride, F, ahi, alo, Lp1, step, flag
  if (first && last) tma_launch_one<T, true, true>(KES_TMA_ARGS);
  else if (first) tma_launch_one<T, true, false>(KES_TMA_ARGS);
  else if (last) tma_launch_one<T, false, true>(KES_TMA_ARGS);
  else tma_launch_one<T, false, false>(KES_TMA_ARGS);
#undef KES_TMA_ARGS
}

template <typename T>
cudaError_t tma_prepare_t(size_t smem) {
  cudaError_t e = cudaSuccess;
  auto set = [&](auto kern) {
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (r != cudaSuccess) e = r;
  };
  set(k_step_tma<T, true, true>);
  set(k_step_tma<T, true, false>);
  set(k_step_tma<T, false, true>);
  set(k_step_tma<T, false, false>);
  return e;
}

}  // namespace

bool tma_shape_fits(bool fp32, const TmaShape& sh) {
  const size_t smem = fp32 ? tma_smem<float>(sh.G, sh.S, sh.wmax) : tma_smem<double>(sh.G, sh.S, sh.wmax);
  return sh.wmax > 0 && smem * sh.ctas_per_sm <= 220 * 1024 && smem <= 200 * 1024;
}

cudaError_t tma_prepare(bool fp32, const TmaShape& sh) {
  const size_t smem = fp32 ? tma_smem<float>(sh.G, sh.S, sh.wmax) : tma_smem<double>(sh.G, sh.S, sh.wmax);
  return fp32 ? tma_prepare_t<float>(smem) : tma_prepare_t<double>(smem);
}

void launch_step_tma_f64(const SellDev& A, const TmaShape& sh, int n_sm, cudaStream_t st, bool first, bool last,
                         const double* x, const double* prev, double* out, double* acc, int64_t acc_stride, int F,
                         const double* alpha, int L, int step, int* flag) {
  tma_dispatch<double>(sh, n_sm, st, first, last, A, x, prev, out, acc, nullptr, nullptr, acc_stride, F, alpha,
                       nullptr, L + 1, step, flag);
  ++g_launches;
}

void launch_step_tma_f32(const SellDev& A, const TmaShape& sh, int n_sm, cudaStream_t st, bool first, bool last,
                         const float* x, const float* prev, float* out, float* acc_s, float* acc_c, double* acc64,
                         int64_t acc_stride, int F, const float* alpha_hi, const float* alpha_lo, int L, int step,
                         int* flag) {
  tma_dispatch<float>(sh, n_sm, st, first, last, A, x, prev, out, acc_s, acc_c, acc64, acc_stride, F, alpha_hi,
                      alpha_lo, L + 1, step, flag);
  ++g_launches;
}

}  // namespace kes
