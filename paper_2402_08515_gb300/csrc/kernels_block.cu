// Block (SpMM) form of the fused leapfrog step: NB start vectors advance together,
// so each stored matrix entry streamed from HBM serves NB products (Sec. 4, block
// version of the Krylov space; eq. 2stepmethod and eq. disc_filtercoeff per column).
//
// State, previous state, output and accumulators are row-major n_pad x NB: the NB
// values of a row are contiguous (32 B for FP32 and NB = 8, one sector), so the
// gather of x at a column index is one or a few 16-byte vector loads per lane.
// A warp owns a 32-row SELL slice exactly as in the single-vector kernels; the
// values and columns stream evict-first, and every column's sum is formed in the
// same order as the single-vector kernel forms it.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "kes_internal.h"

namespace kes {
namespace {

template <typename T>
__device__ __forceinline__ T ld_cs(const T* p) { return __ldcs(p); }

// Asks the memory system to bring the line holding p into L2; moves nothing into
// registers, so a kernel computes the same with or without it.
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// NB contiguous values at p (16-byte aligned for NB * sizeof(T) >= 16; 32-byte aligned for
// 8 floats) through the read-only path. A row of 8 floats is one 32-byte sector, fetched by
// one 256-bit load (sm_100 and later) instead of two 128-bit ones: the gathers of the SpMM
// step issue half the L1 requests.
template <int NB>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&v)[NB]) {
  if constexpr (NB == 1) {
    v[0] = __ldg(p);
  } else if constexpr (NB == 8) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
  } else if constexpr (NB >= 4) {
#pragma unroll
    for (int q = 0; q < NB / 4; ++q) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p) + q);
      v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
  } else {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x; v[1] = t.y;
  }
}
template <int NB>
__device__ __forceinline__ void load_row(const double* __restrict__ p, double (&v)[NB]) {
  if constexpr (NB == 1) {
    v[0] = __ldg(p);
    return;
  }
#pragma unroll
  for (int q = 0; q < NB / 2; ++q) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p) + q);
    v[2 * q] = t.x; v[2 * q + 1] = t.y;
  }
}
// Coherent loads and stores of one row's NB contiguous values with 8-, 16- or (8 floats)
// 32-byte vector accesses (rows are NB * sizeof(T) aligned): a lane moves its whole row in
// 1-4 instructions instead of NB scalar ones that each touch a separate sector.
template <int NB>
__device__ __forceinline__ void load_plain(const float* p, float (&v)[NB]) {
  if constexpr (NB == 1) {
    v[0] = *p;
  } else if constexpr (NB == 8) {
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p)
                 : "memory");
  } else if constexpr (NB >= 4) {
#pragma unroll
    for (int q = 0; q < NB / 4; ++q) {
      const float4 t = reinterpret_cast<const float4*>(p)[q];
      v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
  } else {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  }
}
template <int NB>
__device__ __forceinline__ void load_plain(const double* p, double (&v)[NB]) {
  if constexpr (NB == 1) {
    v[0] = *p;
    return;
  }
#pragma unroll
  for (int q = 0; q < NB / 2; ++q) {
    const double2 t = reinterpret_cast<const double2*>(p)[q];
    v[2 * q] = t.x; v[2 * q + 1] = t.y;
  }
}
template <int NB>
__device__ __forceinline__ void store_row(float* p, const float (&v)[NB]) {
  if constexpr (NB == 1) {
    *p = v[0];
  } else if constexpr (NB == 8) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
  } else if constexpr (NB >= 4) {
#pragma unroll
    for (int q = 0; q < NB / 4; ++q)
      reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  }
}
template <int NB>
__device__ __forceinline__ void store_row(double* p, const double (&v)[NB]) {
  if constexpr (NB == 1) {
    *p = v[0];
    return;
  }
#pragma unroll
  for (int q = 0; q < NB / 2; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(v[2 * q], v[2 * q + 1]);
}

// One row's NB values read again through an opaque (volatile) load: the accumulation of a
// step re-reads u_{n-1} and u_n after the row sums instead of keeping them in registers
// across the gather loop (the compiler may not merge it with the first read). The rows were
// read a moment before and are normally still in L1 or L2.
template <int NB>
__device__ __forceinline__ void reload_row(const float* p, float (&v)[NB]) {
  if constexpr (NB == 8) {
    load_plain<8>(p, v);  // a volatile 256-bit load already
  } else {
#pragma unroll
    for (int q = 0; q < NB; ++q) asm volatile("ld.global.f32 %0, [%1];" : "=f"(v[q]) : "l"(p + q) : "memory");
  }
}
template <int NB>
__device__ __forceinline__ void reload_row(const double* p, double (&v)[NB]) {
#pragma unroll
  for (int q = 0; q < NB; ++q) asm volatile("ld.global.f64 %0, [%1];" : "=d"(v[q]) : "l"(p + q) : "memory");
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  t = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

__device__ __forceinline__ int32_t ld_idx(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_idx(const int16_t* p) { return __ldcs(reinterpret_cast<const short*>(p)); }

// un[j] += sum_k v[32k] * g[col_k * NB + co + j], j < NH, over the w entries of a row, in
// entry order; col_k = base + c[32k] (absolute int32 columns with base 0, or the 16-bit
// column - row differences with base = row). Two entries' loads are issued together.
template <typename T, int NB, int NH, typename I>
__device__ __forceinline__ void row_sums(T (&un)[NH], const T* __restrict__ vp, const I* __restrict__ cp, int base,
                                         int w, const T* __restrict__ g, int co) {
  int k = 0;
  for (; k + 2 <= w; k += 2) {
    const int32_t c0 = base + ld_idx(cp + k * kSliceC), c1 = base + ld_idx(cp + (k + 1) * kSliceC);
    const T v0 = ld_cs(vp + k * kSliceC), v1 = ld_cs(vp + (k + 1) * kSliceC);
    T x0[NH], x1[NH];
    load_row<NH>(g + static_cast<int64_t>(c0) * NB + co, x0);
    load_row<NH>(g + static_cast<int64_t>(c1) * NB + co, x1);
#pragma unroll
    for (int j = 0; j < NH; ++j) un[j] = fma(v1, x1[j], fma(v0, x0[j], un[j]));
  }
  if (k < w) {
    const int32_t c0 = base + ld_idx(cp + k * kSliceC);
    const T v0 = ld_cs(vp + k * kSliceC);
    T x0[NH];
    load_row<NH>(g + static_cast<int64_t>(c0) * NB + co, x0);
#pragma unroll
    for (int j = 0; j < NH; ++j) un[j] = fma(v0, x0[j], un[j]);
  }
}

// The same sums with the matrix stream software-pipelined: the columns and values of the
// next PB entries are loaded while the PB rows of the current ones are gathered, so each
// slice meets the HBM latency of its index stream about once instead of once per pair
// of entries. The chain is still one FMA per entry in entry order (bitwise the sums of
// row_sums). Entries past w (the last batch of a row) are neither loaded nor summed.
template <typename T, int NB, int NH, int PB, typename I>
__device__ __forceinline__ void row_sums_pipe(T (&un)[NH], const T* __restrict__ vp, const I* __restrict__ cp,
                                              int base, int w, const T* __restrict__ g, int co) {
  // entries past w read column `base` (a valid row) with value 0 and are not summed
  int32_t cn[PB];
  T vn[PB];
#pragma unroll
  for (int j = 0; j < PB; ++j) {
    const bool ok = j < w;
    cn[j] = base + (ok ? ld_idx(cp + j * kSliceC) : 0);
    vn[j] = ok ? ld_cs(vp + j * kSliceC) : T(0);
  }
  for (int k = 0; k < w; k += PB) {
    T xx[PB][NH];
#pragma unroll
    for (int j = 0; j < PB; ++j) load_row<NH>(g + static_cast<int64_t>(cn[j]) * NB + co, xx[j]);
    T vv[PB];
#pragma unroll
    for (int j = 0; j < PB; ++j) vv[j] = vn[j];
#pragma unroll
    for (int j = 0; j < PB; ++j) {
      const bool ok = k + PB + j < w;
      cn[j] = base + (ok ? ld_idx(cp + (k + PB + j) * kSliceC) : 0);
      vn[j] = ok ? ld_cs(vp + (k + PB + j) * kSliceC) : T(0);
    }
#pragma unroll
    for (int j = 0; j < PB; ++j)
      if (k + j < w) {
#pragma unroll
        for (int q = 0; q < NH; ++q) un[q] = fma(vv[j], xx[j][q], un[q]);
      }
  }
}

// g: the rows the sums gather from (x itself for the leapfrog, the fourth-order stage
// otherwise); x seeds each row with 2 u_n - u_{n-1}.
// LPR lanes share a row: LPR = 1 gives a lane a whole row of NB columns and a warp a
// 32-row slice; LPR = 2 gives a lane NB / 2 columns and a warp half a slice (16 rows),
// which halves the registers a thread needs for its columns. Either way every column is
// the same FMA chain in entry order, so the shapes round identically. PB > 0 pipelines the
// matrix stream PB entries ahead (row_sums_pipe); PB = 0 loads entries in pairs.
//
// Accumulation (eq. disc_filtercoeff): a step holds u_{n-1}, u_n and u_{n+1} of its rows in
// registers, so the weighted terms need not reach the accumulators every step. With ACC the
// step adds the last nterm (1-3) of alpha_{n-1} u_{n-1}, alpha_n u_n, alpha_{n+1} u_{n+1}, in
// that order (init: the accumulator starts at the first of them, FP64 form); without ACC it
// leaves the accumulator rows alone. The host runs the accumulation every third step and at
// the last: each term is still added once, in index order, with the same operations, so the
// sums are bitwise those of one term per step, and the accumulator rows (for 8 FP32 columns
// 128 of the step's ~320 bytes per row) move every third step only.
template <typename T, int NB, bool FIRST, bool LAST, bool ACC, int MINB, bool PF, int LPR, int PB>
__global__ void __launch_bounds__(256, MINB)
    k_step_blk(SellDev A, const T* __restrict__ x, const T* __restrict__ g, const T* prev, T* out, T* acc_s,
               T* acc_c, double* acc64, int64_t acc_stride, int F, const T* __restrict__ ahi,
               const T* __restrict__ alo, int Lp1, int step, int cpt, uint32_t coltab, int nterm, int init,
               int* flag) {
  // cpt == 0: every column accumulates with all F weight tables (F accumulators);
  // cpt > 0: column j accumulates only with table min(j / cpt, F - 1) (one accumulator)
  constexpr bool kF32 = std::is_same<T, float>::value;
  constexpr int NH = NB / LPR;            // columns of this lane
  constexpr int kRows = kSliceC / LPR;    // rows of a warp's unit
  static_assert(LPR == 1 || !PF, "the L2 prefetch shapes take whole slices");
  static_assert(ACC || !LAST, "the last step completes the sums");
  const T* val;
  if constexpr (kF32) val = A.val32;
  else val = A.val64;
  const int lane = threadIdx.x & 31;
  const int sub = lane / LPR;             // row within the unit
  const int co = (lane % LPR) * NH;       // first column of this lane
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const int64_t n_units = A.n_slices * LPR;
  // PF: L2 prefetch of a slice's streamed lines (column indices, values, u_{n-1} and, when
  // this step reads them, the accumulator rows), the warp's first slice up front and each
  // next slice while the current one is gathered, so that the dependent index -> gather ->
  // FMA chain meets L2 instead of HBM latency. Every address lies inside the slice's own
  // entries/rows.
  const int nacc = cpt ? 1 : F;
  auto prefetch_slice = [&](int64_t sn) {
    if (sn >= A.n_slices) return;
    const int64_t bn = A.slice_ptr[sn];
    const int wn = static_cast<int>((A.slice_ptr[sn + 1] - bn) >> 5);
    constexpr int kValLines = static_cast<int>(sizeof(T)) / 4;  // 128-byte lines per 32 values
    for (int l = lane; l < wn; l += 32) prefetch_l2(A.col + bn + static_cast<int64_t>(l) * kSliceC);
    for (int l = lane; l < wn * kValLines; l += 32)
      prefetch_l2(val + bn + static_cast<int64_t>(l) * (128 / static_cast<int>(sizeof(T))));
    constexpr int kRowLines = kSliceC * NB * static_cast<int>(sizeof(T)) / 128;  // lines of 32 rows x NB
    if (lane < kRowLines) {
      const int64_t off = sn * kSliceC * NB + lane * (128 / static_cast<int>(sizeof(T)));
      if (!FIRST) prefetch_l2(prev + off);
      if (ACC && !init)
        for (int f = 0; f < nacc; ++f) {
          prefetch_l2(acc_s + f * acc_stride + off);
          if (kF32) prefetch_l2(acc_c + f * acc_stride + off);
        }
    }
  };
  const int64_t u0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if constexpr (PF) prefetch_slice(u0);
  for (int64_t u = u0; u < n_units; u += nwarps) {
    if constexpr (PF) prefetch_slice(u + nwarps);
    const int64_t s = u / LPR;
    const int rs = static_cast<int>(u % LPR) * kRows + sub;  // row within the slice
    const int64_t beg = A.slice_ptr[s];
    const int w = static_cast<int>((A.slice_ptr[s + 1] - beg) >> 5);
    const int64_t mesh = A.slice_mesh ? A.slice_mesh[s] : 0;
    const T* vp = val + beg + rs;
    const int64_t row = s * kSliceC + rs;
    const int64_t ro = row * NB + co;  // this lane's values in a row-major block
    T xi[NH], pi[NH], un[NH];
    load_plain<NH>(x + ro, xi);
    if constexpr (FIRST) {
#pragma unroll
      for (int j = 0; j < NH; ++j) pi[j] = xi[j];
    } else {
      load_plain<NH>(prev + ro, pi);
    }
    // u_{n+1} = (2 u_n - u_{n-1}) + A u_n: one FMA chain per column in entry order,
    // seeded like the single-vector kernels, so every column rounds like them
#pragma unroll
    for (int j = 0; j < NH; ++j) {
      if constexpr (kF32) un[j] = __fsub_rn(__fmul_rn(2.0f, xi[j]), pi[j]);
      else un[j] = A.fold2 ? -pi[j] : 2.0 * xi[j] - pi[j];  // A.fold2: 2 x_j is in the diagonal
    }
    if constexpr (PB > 0) {
      if (A.dcol) row_sums_pipe<T, NB, NH, PB>(un, vp, A.dcol + beg + rs, static_cast<int>(row), w, g, co);
      else row_sums_pipe<T, NB, NH, PB>(un, vp, A.col + beg + rs, 0, w, g, co);
    } else {
      if (A.dcol) row_sums<T, NB, NH>(un, vp, A.dcol + beg + rs, static_cast<int>(row), w, g, co);
      else row_sums<T, NB, NH>(un, vp, A.col + beg + rs, 0, w, g, co);
    }
    if constexpr (!ACC) store_row<NH>(out + ro, un);
    if constexpr (ACC) {
      bool bad = false;
      const int tf = static_cast<int>(mesh) * F;
      for (int f = 0; f < nacc; ++f) {
        const int64_t at = f * acc_stride + ro;
        // term t = 0, 1, 2 is alpha_m u_m, m = step - 1 + t, with u_{n-1}, u_n read again
        // (not kept in registers across the gather loop) and u_{n+1} from the row sums;
        // column j's weight comes from its table (cpt > 0: the column's; padding columns
        // take the last one). One term at a time, so that only one term's weights are live.
        auto term_row = [&](int t, T (&uu)[NH]) {
          if (t == 0) {
            if constexpr (FIRST) reload_row<NH>(x + ro, uu);
            else reload_row<NH>(prev + ro, uu);
          } else if (t == 1) {
            reload_row<NH>(x + ro, uu);
          } else {
#pragma unroll
            for (int j = 0; j < NH; ++j) uu[j] = un[j];
          }
        };
        // table of column j; the columns of one table are contiguous, so a term's weights are
        // loaded once per table the lane's columns meet (once when cpt == 0)
        auto table_of = [&](int j) { return cpt ? static_cast<int>((coltab >> (4 * (co + j))) & 15u) : f; };
        if constexpr (kF32) {
          float as[NH], ac[NH];
          load_plain<NH>(acc_s + at, as);
          load_plain<NH>(acc_c + at, ac);
          // (s, c) += alpha_m u_m with alpha_m = hi + lo: the sum's rounding error (Knuth's
          // two-sum), the product's (an FMA) and the low weight's term go to c
#pragma unroll 1
          for (int t = 3 - nterm; t < 3; ++t) {
            float uu[NH];
            term_row(t, uu);
            int tb = -1;
            float h = 0.f, l = 0.f;
#pragma unroll
            for (int j = 0; j < NH; ++j) {
              if (table_of(j) != tb) {
                tb = table_of(j);
                const int ai = (tf + tb) * Lp1 + step - 1 + t;
                h = ahi[ai];
                l = alo[ai];
              }
              const float p = __fmul_rn(h, uu[j]);
              const float pe = fmaf(l, uu[j], fmaf(h, uu[j], -p));
              float sn, e;
              two_sum(as[j], p, sn, e);
              ac[j] = __fadd_rn(ac[j], __fadd_rn(e, pe));
              as[j] = sn;
            }
          }
          if constexpr (LAST) {
            double v64[NH];
#pragma unroll
            for (int j = 0; j < NH; ++j) {
              v64[j] = static_cast<double>(as[j]) + static_cast<double>(ac[j]);
              bad |= !isfinite(v64[j]);
            }
            store_row<NH>(acc64 + at, v64);
          } else {
            store_row<NH>(acc_s + at, as);
            store_row<NH>(acc_c + at, ac);
          }
        } else {
          double na[NH];
          const int t0 = 3 - nterm;
          if (!init) load_plain<NH>(acc_s + at, na);
#pragma unroll 1
          for (int t = t0; t < 3; ++t) {
            double uu[NH];
            term_row(t, uu);
            const bool fresh = init && t == t0;  // the accumulator starts at its first term's product
            int tb = -1;
            double h = 0.0;
#pragma unroll
            for (int j = 0; j < NH; ++j) {
              if (table_of(j) != tb) {
                tb = table_of(j);
                h = ahi[(tf + tb) * Lp1 + step - 1 + t];
              }
              na[j] = fresh ? h * uu[j] : fma(h, uu[j], na[j]);
            }
          }
          if constexpr (LAST) {
#pragma unroll
            for (int j = 0; j < NH; ++j) bad |= !isfinite(na[j]);
          }
          store_row<NH>(acc_s + at, na);
        }
      }
      // after every read of u_{n-1}: out may share its storage
      if constexpr (!LAST) store_row<NH>(out + ro, un);
      if (LAST && bad) atomicOr(flag, 1);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Block step in FP32 pairs (double-float arithmetic): every step value, state value and
// row sum is an unevaluated sum hi + lo of two FP32 numbers. A product a x of two pairs is
// taken as ph = fl(a_hi x_hi) plus the error of that product (an FMA gives it exactly) and
// the cross terms a_hi x_lo + a_lo x_hi; the row sum adds ph by Knuth's two-sum and keeps
// the rounding errors and the small terms in a compensation word, normalised at the end of
// the row. This carries a significand of about 48 bits with FP32 instructions only (the
// FP64 units of GB300 issue about two FMAs per clock per SM). Same recurrence and order as
// the other step kernels (eq. 2stepmethod; the values hold A + 2I when fold2), the weighted
// terms added to the compensated FP32 accumulator every third step like k_step_blk.
// kX2Lpr lanes per row: a lane owns NH = NB / kX2Lpr columns, a warp 32 / kX2Lpr rows.
// NH (hi, lo) pairs of one row: coherent and read-only-path loads, and the store
template <int NH>
__device__ __forceinline__ void load_pairs(const float2* p, float (&h)[NH], float (&l)[NH]) {
  float v[2 * NH];
  load_plain<2 * NH>(reinterpret_cast<const float*>(p), v);
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    h[j] = v[2 * j];
    l[j] = v[2 * j + 1];
  }
}
template <int NH>
__device__ __forceinline__ void load_pairs_nc(const float2* __restrict__ p, float (&h)[NH], float (&l)[NH]) {
  float v[2 * NH];
  load_row<2 * NH>(reinterpret_cast<const float*>(p), v);
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    h[j] = v[2 * j];
    l[j] = v[2 * j + 1];
  }
}
template <int NH>
__device__ __forceinline__ void store_pairs(float2* p, const float (&h)[NH], const float (&l)[NH]) {
  float v[2 * NH];
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    v[2 * j] = h[j];
    v[2 * j + 1] = l[j];
  }
  store_row<2 * NH>(reinterpret_cast<float*>(p), v);
}

// (sh, sl) += (ah + al)(xh + xl), the product's low-order terms and the sum's rounding error
// into sl
__device__ __forceinline__ void pair_fma(float ah, float al, float xh, float xl, float& sh, float& sl) {
  const float ph = __fmul_rn(ah, xh);
  float pe = fmaf(ah, xh, -ph);
  pe = fmaf(ah, xl, pe);
  pe = fmaf(al, xh, pe);
  float t, e;
  two_sum(sh, ph, t, e);
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(e, pe));
}

// Lanes per row and resident blocks per SM of the FP32-pair step.
constexpr int kX2Lpr = 2, kX2MinBlocks = 4;

template <int NB, bool FIRST, bool LAST, bool ACC>
__global__ void __launch_bounds__(256, kX2MinBlocks)
    k_step_x2(SellDev A, const float2* __restrict__ val2, const float2* __restrict__ x, const float2* prev,
              float2* out, float* acc_s, float* acc_c, double* acc64, int64_t acc_stride, int F,
              const float* __restrict__ ahi, const float* __restrict__ alo, int Lp1, int step, int cpt,
              uint32_t coltab, int nterm, int* flag) {
  constexpr int LPR = NB >= kX2Lpr ? kX2Lpr : NB;
  constexpr int NH = NB / LPR;            // columns of this lane
  constexpr int kRows = kSliceC / LPR;    // rows of a warp's unit
  static_assert(ACC || !LAST, "the last step completes the sums");
  const int lane = threadIdx.x & 31;
  const int sub = lane / LPR;             // row within the unit
  const int co = (lane % LPR) * NH;       // first column of this lane
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const int64_t n_units = A.n_slices * LPR;
  const int nacc = cpt ? 1 : F;
  for (int64_t u = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; u < n_units; u += nwarps) {
    const int64_t s = u / LPR;
    const int rs = static_cast<int>(u % LPR) * kRows + sub;  // row within the slice
    const int64_t beg = A.slice_ptr[s];
    const int w = static_cast<int>((A.slice_ptr[s + 1] - beg) >> 5);
    const int64_t mesh = A.slice_mesh ? A.slice_mesh[s] : 0;
    const int64_t row = s * kSliceC + rs;
    const int64_t ro = row * NB + co;
    float sh[NH], sl[NH];
    {
      float xh[NH], xl[NH], ph[NH], pl[NH];
      load_pairs<NH>(x + ro, xh, xl);
      if constexpr (FIRST) {
#pragma unroll
        for (int j = 0; j < NH; ++j) {
          ph[j] = xh[j];
          pl[j] = xl[j];
        }
      } else {
        load_pairs<NH>(prev + ro, ph, pl);
      }
      // seed: -u_{n-1} when the values hold A + 2I, else 2 u_n - u_{n-1} (2 x is exact)
#pragma unroll
      for (int j = 0; j < NH; ++j) {
        if (A.fold2) {
          sh[j] = -ph[j];
          sl[j] = -pl[j];
        } else {
          float t, e;
          two_sum(__fmul_rn(2.0f, xh[j]), -ph[j], t, e);
          sh[j] = t;
          sl[j] = __fadd_rn(e, __fsub_rn(__fmul_rn(2.0f, xl[j]), pl[j]));
        }
      }
    }
    // the row's entries in order, two at a time
    const float2* vp = val2 + beg + rs;
    const int base = A.dcol ? static_cast<int>(row) : 0;
    int k = 0;
    for (; k + 2 <= w; k += 2) {
      const int32_t c0 = base + (A.dcol ? ld_idx(A.dcol + beg + rs + k * kSliceC) : ld_idx(A.col + beg + rs + k * kSliceC));
      const int32_t c1 = base + (A.dcol ? ld_idx(A.dcol + beg + rs + (k + 1) * kSliceC)
                                        : ld_idx(A.col + beg + rs + (k + 1) * kSliceC));
      const float2 v0 = __ldcs(vp + k * kSliceC), v1 = __ldcs(vp + (k + 1) * kSliceC);
      float h0[NH], l0[NH], h1[NH], l1[NH];
      load_pairs_nc<NH>(x + static_cast<int64_t>(c0) * NB + co, h0, l0);
      load_pairs_nc<NH>(x + static_cast<int64_t>(c1) * NB + co, h1, l1);
#pragma unroll
      for (int j = 0; j < NH; ++j) {
        pair_fma(v0.x, v0.y, h0[j], l0[j], sh[j], sl[j]);
        pair_fma(v1.x, v1.y, h1[j], l1[j], sh[j], sl[j]);
      }
    }
    if (k < w) {
      const int32_t c0 = base + (A.dcol ? ld_idx(A.dcol + beg + rs + k * kSliceC) : ld_idx(A.col + beg + rs + k * kSliceC));
      const float2 v0 = __ldcs(vp + k * kSliceC);
      float h0[NH], l0[NH];
      load_pairs_nc<NH>(x + static_cast<int64_t>(c0) * NB + co, h0, l0);
#pragma unroll
      for (int j = 0; j < NH; ++j) pair_fma(v0.x, v0.y, h0[j], l0[j], sh[j], sl[j]);
    }
    // u_{n+1} normalised: hi = fl(sh + sl), lo = the rest
    float uh[NH], ul[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) two_sum(sh[j], sl[j], uh[j], ul[j]);
    if constexpr (!ACC) store_pairs<NH>(out + ro, uh, ul);
    if constexpr (ACC) {
      bool bad = false;
      for (int f = 0; f < nacc; ++f) {
        const int64_t at = f * acc_stride + ro;
        auto table_of = [&](int j) { return cpt ? static_cast<int>((coltab >> (4 * (co + j))) & 15u) : f; };
        float as[NH], ac[NH];
        load_plain<NH>(acc_s + at, as);
        load_plain<NH>(acc_c + at, ac);
#pragma unroll 1
        for (int t = 3 - nterm; t < 3; ++t) {
          float th[NH], tl[NH];
          if (t == 0) {
            if constexpr (FIRST) load_pairs<NH>(x + ro, th, tl);
            else load_pairs<NH>(prev + ro, th, tl);
          } else if (t == 1) {
            load_pairs<NH>(x + ro, th, tl);
          } else {
#pragma unroll
            for (int j = 0; j < NH; ++j) {
              th[j] = uh[j];
              tl[j] = ul[j];
            }
          }
          int tb = -1;
          float h = 0.f, l = 0.f;
#pragma unroll
          for (int j = 0; j < NH; ++j) {
            if (table_of(j) != tb) {
              tb = table_of(j);
              const int ai = (static_cast<int>(mesh) * F + tb) * Lp1 + step - 1 + t;
              h = ahi[ai];
              l = alo[ai];
            }
            pair_fma(h, l, th[j], tl[j], as[j], ac[j]);
          }
        }
        if constexpr (LAST) {
          double v64[NH];
#pragma unroll
          for (int j = 0; j < NH; ++j) {
            v64[j] = static_cast<double>(as[j]) + static_cast<double>(ac[j]);
            bad |= !isfinite(v64[j]);
          }
          store_row<NH>(acc64 + at, v64);
        } else {
          store_row<NH>(acc_s + at, as);
          store_row<NH>(acc_c + at, ac);
        }
      }
      // after every read of u_{n-1}: out may share its storage
      if constexpr (!LAST) store_pairs<NH>(out + ro, uh, ul);
      if (LAST && bad) atomicOr(flag, 1);
    }
  }
}

// FP32-pair start for nb columns: x2 = r split as hi + lo, and the compensated accumulators
// set to alpha_f[0] r as k_init_f32 sets them.
__global__ void k_init_x2(int64_t count, int nb, const double* __restrict__ r, float2* __restrict__ x2,
                          float* __restrict__ acc_s, float* __restrict__ acc_c, int64_t acc_stride, int F,
                          const double* __restrict__ alpha, int Lp1, const int32_t* __restrict__ slice_mesh,
                          int cpt) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double ri = r[i];
    const float hi = static_cast<float>(ri);
    x2[i] = make_float2(hi, static_cast<float>(ri - static_cast<double>(hi)));
    const int64_t mesh = slice_mesh ? slice_mesh[(i / nb) / kSliceC] : 0;
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

// FP64 step values split into FP32 pairs, hi = fl(v), lo = fl(v - hi)
__global__ void k_split_values(int64_t count, const double* __restrict__ v, float2* __restrict__ v2) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double a = v[i];
    const float hi = static_cast<float>(a);
    v2[i] = make_float2(hi, static_cast<float>(a - static_cast<double>(hi)));
  }
}

// Launch shapes of the block kernels: minimum resident 256-thread blocks per SM, whether
// the slices are prefetched into L2, lanes per row, entries of the pipelined matrix stream
// (0: pairs, not pipelined). (Copying each slice's accumulator rows into shared memory with
// cp.async when the slice starts was measured as well: 186-201 us against 173 us for
// shape 13 on the 12-mesh batch, so it is not offered.)
#define KES_BLK_VARIANTS(X)                                                                         \
  X(0, 1, false, 1, 0) X(1, 2, false, 1, 0) X(2, 3, false, 1, 0) X(3, 4, false, 1, 0)              \
  X(4, 1, true, 1, 0) X(5, 2, true, 1, 0) X(6, 3, true, 1, 0) X(7, 4, true, 1, 0)                   \
  X(8, 4, false, 2, 0) X(9, 5, false, 2, 0) X(10, 6, false, 2, 0) X(11, 4, false, 1, 2)             \
  X(12, 3, false, 1, 4) X(13, 4, false, 1, 4) X(14, 2, false, 1, 8) X(15, 6, false, 2, 4)           \
  X(16, 4, false, 2, 8)

template <typename T, int NB, int MINB, bool PF, int LPR, int PB>
void blk_impl(int grid, int block, cudaStream_t st, bool first, bool last, const SellDev& A, const T* x,
              const T* g, const T* prev, T* out, T* acc_s, T* acc_c, double* acc64, int64_t acc_stride, int F, const T* ahi,
              const T* alo, int Lp1, int step, int cpt, uint32_t coltab, int nterm, int init, int* flag) {
#define KES_BLK_ARGS \
  A, x, g, prev, out, acc_s, acc_c, acc64, acc_stride, F, ahi, alo, Lp1, step, cpt, coltab, nterm, init, flag
#define KES_BLK(FI, LA, AC) k_step_blk<T, NB, FI, LA, AC, MINB, PF, LPR, PB><<<grid, block, 0, st>>>(KES_BLK_ARGS)
  if (first && last) KES_BLK(true, true, true);
  else if (last) KES_BLK(false, true, true);
  else if (first && nterm) KES_BLK(true, false, true);
  else if (first) KES_BLK(true, false, false);
  else if (nterm) KES_BLK(false, false, true);
  else KES_BLK(false, false, false);
#undef KES_BLK
#undef KES_BLK_ARGS
}

template <typename T>
void blk_dispatch(const LaunchCfg& cfg, int NB, cudaStream_t st, bool first, bool last, const SellDev& A,
                  const T* x, const T* g, const T* prev, T* out, T* acc_s, T* acc_c, double* acc64, int64_t acc_stride, int F,
                  const T* ahi, const T* alo, int Lp1, int step, int cpt, int nterm, int init, int* flag) {
  // cpt > 0: weight table min(c / cpt, F - 1) of each column c, 4 bits per column (at most
  // one table per column there, so F <= NB <= 8), passed as a kernel parameter
  uint32_t coltab = 0;
  if (cpt > 0)
    for (int c = 0; c < NB; ++c) coltab |= static_cast<uint32_t>(std::min(c / cpt, F - 1)) << (4 * c);
  // a block of 256 threads is 8 warps; a warp takes a slice (or half a slice, LPR = 2)
  int lpr = 1;
#define X(ID, M, P, R, B) \
  if (cfg.variant_blk == ID) lpr = R;
  KES_BLK_VARIANTS(X)
#undef X
  const int64_t need = (A.n_slices * lpr + 7) / 8;
  const int grid = static_cast<int>(need < cfg.grid_blk ? need : cfg.grid_blk);
#define KES_CALL(NBV, M, P, R, B)                                                                             \
  blk_impl<T, NBV, M, P, R, B>(grid, 256, st, first, last, A, x, g, prev, out, acc_s, acc_c, acc64, acc_stride, F, \
                               ahi, alo, Lp1, step, cpt, coltab, nterm, init, flag)
#define X(ID, M, P, R, B)                         \
  case ID:                                        \
    if (NB == 2) KES_CALL(2, M, P, R, B);         \
    else if (NB == 4) KES_CALL(4, M, P, R, B);    \
    else KES_CALL(8, M, P, R, B);                 \
    break;
  switch (cfg.variant_blk) {
    KES_BLK_VARIANTS(X)
    default: break;
  }
#undef X
#undef KES_CALL
}

// Stage of the fourth-order modified-equation leapfrog (Remark 2.4): v = u + A u / 12
// for NB row-major columns (NB = 1: a plain vector), A = -tau^2 M^{-1} S in the SELL
// layout, one warp per 32-row slice as in the step kernels. The step kernel then
// gathers A v = -tau^2 K u + (tau^4 / 12) K^2 u (K = M^{-1} S).
template <typename T, int NB>
__global__ void __launch_bounds__(256) k_stage4(SellDev A, const T* __restrict__ x, T* __restrict__ v) {
  constexpr bool kF32 = std::is_same<T, float>::value;
  const T* val;
  if constexpr (kF32) val = A.val32;
  else val = A.val64;
  const T twelfth = T(1) / T(12);
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < A.n_slices;
       s += nwarps) {
    const int64_t beg = A.slice_ptr[s];
    const int w = static_cast<int>((A.slice_ptr[s + 1] - beg) >> 5);
    const T* vp = val + beg + lane;
    const int64_t row = s * kSliceC + lane;
    T acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = T(0);
    if (A.dcol) row_sums<T, NB, NB>(acc, vp, A.dcol + beg + lane, static_cast<int>(row), w, x, 0);
    else row_sums<T, NB, NB>(acc, vp, A.col + beg + lane, 0, w, x, 0);
    T xi[NB];
    if constexpr (NB == 1) xi[0] = x[row];
    else load_plain<NB>(x + row * NB, xi);
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = fma(acc[j], twelfth, xi[j]);
    if constexpr (NB == 1) v[row] = acc[0];
    else store_row<NB>(v + row * NB, acc);
  }
}

template <typename T>
void stage4_dispatch(const SellDev& A, int n_sm, cudaStream_t st, int NB, const T* x, T* v) {
  const int64_t need = (A.n_slices + 7) / 8;  // 8 warps of 256 threads, one slice each
  const int64_t cap = static_cast<int64_t>(n_sm) * 8;
  const int grid = static_cast<int>(need < cap ? (need > 0 ? need : 1) : cap);
  if (NB == 1) k_stage4<T, 1><<<grid, 256, 0, st>>>(A, x, v);
  else if (NB == 2) k_stage4<T, 2><<<grid, 256, 0, st>>>(A, x, v);
  else if (NB == 4) k_stage4<T, 4><<<grid, 256, 0, st>>>(A, x, v);
  else k_stage4<T, 8><<<grid, 256, 0, st>>>(A, x, v);
}

template <typename T, int NB, int M, bool P, int R, int B>
int occ_one(int block) {
  int nb = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_blk<T, NB, false, false, true, M, P, R, B>, block, 0) ==
                 cudaSuccess
             ? nb
             : 0;
}

__global__ void k_gather_rows(const double* __restrict__ src, int64_t ld_src, int ncols,
                              const int32_t* __restrict__ row_src, int64_t n_valid, double* __restrict__ dst,
                              int NB, int64_t n_pad) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n_pad * NB;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = t / NB;
    const int j = static_cast<int>(t % NB);
    const int64_t r = row_src ? row_src[i] : (i < n_valid ? i : -1);
    dst[t] = (j < ncols && r >= 0) ? src[j * ld_src + r] : 0.0;
  }
}

__global__ void k_scatter_rows(const double* __restrict__ src, int NB, int ncols,
                               const int32_t* __restrict__ row_src, int64_t n_valid, double* __restrict__ dst,
                               int64_t ld_dst, int64_t n_pad) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n_pad * NB;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = t / NB;
    const int j = static_cast<int>(t % NB);
    const int64_t r = row_src ? row_src[i] : (i < n_valid ? i : -1);
    if (j < ncols && r >= 0) dst[j * ld_dst + r] = src[t];
  }
}

__global__ void k_pack_basis(const double* __restrict__ B, int64_t ldb, const int32_t* __restrict__ colsel,
                             const int32_t* __restrict__ slice_mesh, double* __restrict__ stage, int NB,
                             int64_t n_pad) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n_pad * NB;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = t / NB;
    const int j = static_cast<int>(t % NB);
    const int mesh = slice_mesh ? slice_mesh[i / kSliceC] : 0;
    const int c = colsel[mesh * NB + j];
    stage[t] = c >= 0 ? B[c * ldb + i] : 0.0;
  }
}

__global__ void k_unpack_block(const double* __restrict__ stage, int NB, double* __restrict__ Wc, int64_t n_pad) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n_pad * NB;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = t / NB;
    const int j = static_cast<int>(t % NB);
    Wc[j * n_pad + i] = stage[t];
  }
}

int elem_grid(int64_t count) {
  const int64_t b = (count + 255) / 256;
  return static_cast<int>(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

int blk_variant_count() {
  int n = 0;
#define X(ID, M, P, R, B) ++n;
  KES_BLK_VARIANTS(X)
#undef X
  return n;
}

int blk_blocks_per_sm(bool fp32, int NB, int variant, int block) {
  int nb = 0;
#define X(ID, M, P, R, B)                                                                           \
  case ID:                                                                                          \
    if (fp32)                                                                                       \
      nb = NB == 2 ? occ_one<float, 2, M, P, R, B>(block)                                           \
                   : NB == 4 ? occ_one<float, 4, M, P, R, B>(block) : occ_one<float, 8, M, P, R, B>(block); \
    else                                                                                            \
      nb = NB == 2 ? occ_one<double, 2, M, P, R, B>(block)                                          \
                   : NB == 4 ? occ_one<double, 4, M, P, R, B>(block) : occ_one<double, 8, M, P, R, B>(block); \
    break;
  switch (variant) {
    KES_BLK_VARIANTS(X)
    default: break;
  }
#undef X
  return nb > 0 ? nb : 1;
}

void launch_step_blk_f64(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, int NB, bool first, bool last,
                         const double* x, const double* g, const double* prev, double* out, double* acc,
                         int64_t acc_stride, int F, const double* alpha, int L, int step, int cpt, int nterm,
                         bool init, int* flag) {
  blk_dispatch<double>(cfg, NB, st, first, last, A, x, g, prev, out, acc, nullptr, nullptr, acc_stride, F, alpha,
                       nullptr, L + 1, step, cpt, nterm, init ? 1 : 0, flag);
  ++g_launches;
}

void launch_step_blk_f32(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, int NB, bool first, bool last,
                         const float* x, const float* g, const float* prev, float* out, float* acc_s, float* acc_c,
                         double* acc64, int64_t acc_stride, int F, const float* alpha_hi, const float* alpha_lo,
                         int L, int step, int cpt, int nterm, int* flag) {
  blk_dispatch<float>(cfg, NB, st, first, last, A, x, g, prev, out, acc_s, acc_c, acc64, acc_stride, F, alpha_hi,
                      alpha_lo, L + 1, step, cpt, nterm, 0, flag);
  ++g_launches;
}

void launch_step_x2(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, int NB, bool first, bool last,
                    const float2* val2, const float2* x, const float2* prev, float2* out, float* acc_s, float* acc_c,
                    double* acc64, int64_t acc_stride, int F, const float* alpha_hi, const float* alpha_lo, int L,
                    int step, int cpt, int nterm, int* flag) {
  uint32_t coltab = 0;
  if (cpt > 0)
    for (int c = 0; c < NB; ++c) coltab |= static_cast<uint32_t>(std::min(c / cpt, F - 1)) << (4 * c);
  const int lpr = NB >= kX2Lpr ? kX2Lpr : NB;
  const int64_t need = (A.n_slices * lpr + 7) / 8;  // 8 warps per block, 32 / lpr rows each
  const int64_t cap = static_cast<int64_t>(cfg.n_sm) * kX2MinBlocks;
  const int grid = static_cast<int>(need < cap ? (need > 0 ? need : 1) : cap);
#define KES_X2_ARGS A, val2, x, prev, out, acc_s, acc_c, acc64, acc_stride, F, alpha_hi, alpha_lo, L + 1, step, cpt, coltab, nterm, flag
#define KES_X2(NBV)                                                                               \
  if (last) {                                                                                     \
    if (first) k_step_x2<NBV, true, true, true><<<grid, 256, 0, st>>>(KES_X2_ARGS);               \
    else k_step_x2<NBV, false, true, true><<<grid, 256, 0, st>>>(KES_X2_ARGS);                    \
  } else if (first) {                                                                             \
    if (nterm) k_step_x2<NBV, true, false, true><<<grid, 256, 0, st>>>(KES_X2_ARGS);              \
    else k_step_x2<NBV, true, false, false><<<grid, 256, 0, st>>>(KES_X2_ARGS);                   \
  } else if (nterm) {                                                                             \
    k_step_x2<NBV, false, false, true><<<grid, 256, 0, st>>>(KES_X2_ARGS);                        \
  } else {                                                                                        \
    k_step_x2<NBV, false, false, false><<<grid, 256, 0, st>>>(KES_X2_ARGS);                       \
  }
  if (NB == 2) {
    KES_X2(2)
  } else if (NB == 4) {
    KES_X2(4)
  } else {
    KES_X2(8)
  }
#undef KES_X2
#undef KES_X2_ARGS
  ++g_launches;
}

void launch_init_x2(cudaStream_t st, const SellDev& A, int nb, const double* r64, float2* x2, float* acc_s,
                    float* acc_c, int64_t acc_stride, int F, const double* alpha64, int L, int cpt) {
  const int64_t count = A.n_pad * nb;
  const int64_t blocks = (count + 255) / 256;
  k_init_x2<<<static_cast<int>(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(
      count, nb, r64, x2, acc_s, acc_c, acc_stride, F, alpha64, L + 1, A.slice_mesh, cpt);
  ++g_launches;
}

void launch_split_values(cudaStream_t st, int64_t count, const double* v, float2* v2) {
  const int64_t blocks = (count + 255) / 256;
  k_split_values<<<static_cast<int>(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096), 256, 0, st>>>(count, v, v2);
  ++g_launches;
}

void launch_gather_rows(cudaStream_t st, const double* src, int64_t ld_src, int ncols, const int32_t* row_src,
                        int64_t n_valid, double* dst, int NB, int64_t n_pad) {
  k_gather_rows<<<elem_grid(n_pad * NB), 256, 0, st>>>(src, ld_src, ncols, row_src, n_valid, dst, NB, n_pad);
  ++g_launches;
}

void launch_scatter_rows(cudaStream_t st, const double* src, int NB, int ncols, const int32_t* row_src,
                         int64_t n_valid, double* dst, int64_t ld_dst, int64_t n_pad) {
  k_scatter_rows<<<elem_grid(n_pad * NB), 256, 0, st>>>(src, NB, ncols, row_src, n_valid, dst, ld_dst, n_pad);
  ++g_launches;
}

void launch_stage4_f64(const SellDev& A, int n_sm, cudaStream_t st, int NB, const double* x, double* v) {
  stage4_dispatch<double>(A, n_sm, st, NB, x, v);
  ++g_launches;
}

void launch_stage4_f32(const SellDev& A, int n_sm, cudaStream_t st, int NB, const float* x, float* v) {
  stage4_dispatch<float>(A, n_sm, st, NB, x, v);
  ++g_launches;
}

void launch_pack_basis(cudaStream_t st, const double* B, int64_t ldb, const int32_t* colsel,
                       const int32_t* slice_mesh, double* stage, int NB, int64_t n_pad) {
  k_pack_basis<<<elem_grid(n_pad * NB), 256, 0, st>>>(B, ldb, colsel, slice_mesh, stage, NB, n_pad);
  ++g_launches;
}

void launch_unpack_block(cudaStream_t st, const double* stage, int NB, double* Wc, int64_t n_pad) {
  k_unpack_block<<<elem_grid(n_pad * NB), 256, 0, st>>>(stage, NB, Wc, n_pad);
  ++g_launches;
}

}  // namespace kes
