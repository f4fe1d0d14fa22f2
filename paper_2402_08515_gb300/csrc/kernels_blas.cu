// FP64 vector kernels of the Krylov loop (Algorithm 2.5, orthogonalisation),
// the projection (eq. projevp) and the residuals (eq. res).
//
// All reductions are deterministic: every block writes one partial per
// column in a fixed row order and a second kernel sums the partials in a
// fixed tree order, so repeated runs give bit-identical results.
#include <cuda_runtime.h>

#include "kes_internal.h"

namespace kes {
namespace {

constexpr int kThreads = 256;
constexpr int kGroup = 8;  // columns per block in the multi-column kernels

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduces G per-thread values over the block; thread 0 of warp 0 ends with the sums in out[].
template <int G>
__device__ __forceinline__ void block_sum(double (&v)[G], double (&out)[G]) {
  __shared__ double sh[G][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const double s = warp_sum(v[g]);
    if (lane == 0) sh[g][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      double s = lane < kThreads / 32 ? sh[g][lane] : 0.0;
      out[g] = warp_sum(s);
    }
  }
}

// partial[j * nblk + blk] = sum over this block's rows of B[j*ldb + i] * w[i] * v[i]
__global__ void __launch_bounds__(kThreads) k_mdot_partial(const double* __restrict__ B, int64_t ldb, int k,
                                                           const double* __restrict__ v,
                                                           const double* __restrict__ w, int64_t n,
                                                           double* __restrict__ partial) {
  const int j0 = blockIdx.y * kGroup;
  double acc[kGroup];
#pragma unroll
  for (int g = 0; g < kGroup; ++g) acc[g] = 0.0;
  const int ng = min(kGroup, k - j0);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads) {
    const double wv = w ? w[i] * v[i] : v[i];
#pragma unroll
    for (int g = 0; g < kGroup; ++g)
      if (g < ng) acc[g] = fma(B[(j0 + g) * ldb + i], wv, acc[g]);
  }
  double tot[kGroup];
  block_sum<kGroup>(acc, tot);
  if (threadIdx.x == 0)
    for (int g = 0; g < ng; ++g) partial[static_cast<int64_t>(j0 + g) * gridDim.x + blockIdx.x] = tot[g];
}

// out[j] = sum_b partial[j * nblk + b]
__global__ void __launch_bounds__(kThreads) k_reduce_partial(const double* __restrict__ partial, int nblk,
                                                             double* __restrict__ out) {
  const int j = blockIdx.x;
  double v[1] = {0.0};
  for (int b = threadIdx.x; b < nblk; b += kThreads) v[0] += partial[static_cast<int64_t>(j) * nblk + b];
  double tot[1];
  block_sum<1>(v, tot);
  if (threadIdx.x == 0) out[j] = tot[0];
}

__global__ void __launch_bounds__(kThreads) k_gemv_sub(double* __restrict__ v, const double* __restrict__ B,
                                                       int64_t ldb, int k, const double* __restrict__ h,
                                                       int64_t n) {
  extern __shared__ double sh_h[];
  for (int j = threadIdx.x; j < k; j += kThreads) sh_h[j] = h[j];
  __syncthreads();
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads) {
    double s0 = 0.0, s1 = 0.0;
    int j = 0;
    for (; j + 2 <= k; j += 2) {
      s0 = fma(B[j * ldb + i], sh_h[j], s0);
      s1 = fma(B[(j + 1) * ldb + i], sh_h[j + 1], s1);
    }
    if (j < k) s0 = fma(B[j * ldb + i], sh_h[j], s0);
    v[i] -= s0 + s1;
  }
}

__global__ void k_scale_rsqrt(const double* __restrict__ v, const double* __restrict__ nrm2,
                              double* __restrict__ dst, double* __restrict__ dst2, int64_t n) {
  const double nrm = sqrt(nrm2[0]);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double x = v[i] / nrm;
    dst[i] = x;
    if (dst2) dst2[i] = x;
  }
}

// Ritz residual partial sums for Ritz vectors j0 .. j0+kGroup-1:
// partial[j * nblk + blk] = sum_i (sx_j - theta_j m_i x_j)^2, partial[(p + j) * nblk + blk] = sum_i (m_i x_j)^2
__global__ void __launch_bounds__(kThreads) k_ritz_residual(const double* __restrict__ B,
                                                            const double* __restrict__ SB, int64_t ldb, int k,
                                                            const double* __restrict__ Y,
                                                            const double* __restrict__ theta, int p,
                                                            const double* __restrict__ m, int64_t n,
                                                            double* __restrict__ partial) {
  extern __shared__ double sY[];  // k x kGroup
  const int j0 = blockIdx.y * kGroup;
  const int ng = min(kGroup, p - j0);
  for (int t = threadIdx.x; t < k * kGroup; t += kThreads) {
    const int l = t / kGroup, g = t % kGroup;
    sY[t] = g < ng ? Y[static_cast<int64_t>(j0 + g) * k + l] : 0.0;
  }
  __syncthreads();
  double th[kGroup];
#pragma unroll
  for (int g = 0; g < kGroup; ++g) th[g] = g < ng ? theta[j0 + g] : 0.0;
  double rr[kGroup], mm[kGroup];
#pragma unroll
  for (int g = 0; g < kGroup; ++g) rr[g] = mm[g] = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads) {
    double x[kGroup], sx[kGroup];
#pragma unroll
    for (int g = 0; g < kGroup; ++g) x[g] = sx[g] = 0.0;
    for (int l = 0; l < k; ++l) {
      const double b = B[l * ldb + i], sb = SB[l * ldb + i];
#pragma unroll
      for (int g = 0; g < kGroup; ++g) {
        x[g] = fma(b, sY[l * kGroup + g], x[g]);
        sx[g] = fma(sb, sY[l * kGroup + g], sx[g]);
      }
    }
    const double mi = m[i];
#pragma unroll
    for (int g = 0; g < kGroup; ++g) {
      const double mx = mi * x[g];
      const double r = sx[g] - th[g] * mx;
      rr[g] = fma(r, r, rr[g]);
      mm[g] = fma(mx, mx, mm[g]);
    }
  }
  double trr[kGroup], tmm[kGroup];
  block_sum<kGroup>(rr, trr);
  __syncthreads();
  block_sum<kGroup>(mm, tmm);
  if (threadIdx.x == 0)
    for (int g = 0; g < ng; ++g) {
      partial[static_cast<int64_t>(j0 + g) * gridDim.x + blockIdx.x] = trr[g];
      partial[static_cast<int64_t>(p + j0 + g) * gridDim.x + blockIdx.x] = tmm[g];
    }
}

__global__ void __launch_bounds__(kThreads) k_gemm_bx(const double* __restrict__ B, int64_t ldb, int k,
                                                      const double* __restrict__ Y, int p,
                                                      double* __restrict__ X, int64_t ldx, int64_t n) {
  extern __shared__ double sY[];
  const int j0 = blockIdx.y * kGroup;
  const int ng = min(kGroup, p - j0);
  for (int t = threadIdx.x; t < k * kGroup; t += kThreads) {
    const int l = t / kGroup, g = t % kGroup;
    sY[t] = g < ng ? Y[static_cast<int64_t>(j0 + g) * k + l] : 0.0;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads) {
    double x[kGroup];
#pragma unroll
    for (int g = 0; g < kGroup; ++g) x[g] = 0.0;
    for (int l = 0; l < k; ++l) {
      const double b = B[l * ldb + i];
#pragma unroll
      for (int g = 0; g < kGroup; ++g) x[g] = fma(b, sY[l * kGroup + g], x[g]);
    }
    for (int g = 0; g < ng; ++g) X[(j0 + g) * ldx + i] = x[g];
  }
}

__global__ void k_permute(const double* __restrict__ src, double* __restrict__ dst,
                          const int32_t* __restrict__ perm, int64_t n, bool gather) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (gather) dst[i] = src[perm[i]];
    else dst[perm[i]] = src[i];
  }
}

__global__ void k_scale(const double* __restrict__ src, double s, double* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[i] = src[i] * s;
}

// Kernels whose dynamic shared memory grows with the basis size k (k x 8 doubles of Ritz
// coefficients, next to their static shared memory) may need more than the default 48 KB
// per block: raise the kernel's limit
// to what the launch asks for (up to the device's opt-in maximum, 227 KB on GB300, which
// bounds k at kMaxProjected). Returns false if the launch cannot get that much; the launch
// then fails and the caller's launch check reports it.
bool allow_dynamic_smem(const void* fn, size_t bytes) {
  cudaFuncAttributes attr{};
  if (cudaFuncGetAttributes(&attr, fn) != cudaSuccess) return false;
  if (bytes + attr.sharedSizeBytes <= 48 * 1024) return true;  // within the default limit
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  if (bytes + attr.sharedSizeBytes > static_cast<size_t>(optin)) return false;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)) ==
         cudaSuccess;
}

int rows_grid(int64_t n, int cap) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return static_cast<int>(b < cap ? (b > 0 ? b : 1) : cap);
}

// The batched kernels: the 1D grid is the concatenation of the jobs' blocks; a block finds
// its job by binary search over the jobs' first blocks, then works as a block of that
// job's own launch would (rows strided by the job's nblk), so the sums are the same.
template <typename J>
__device__ __forceinline__ int job_of(const J* __restrict__ jobs, int njobs, int64_t bid) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].first <= bid) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Batched M-inner products h_j = sum_i B[j*ldb + i] w_i v_i (Algorithm 2.5, the M-inner
// product of the orthogonalisation). A block owns kBlockRows consecutive rows of its job
// and each of its 8 warps kWarpRows of them (16 slabs of 32 rows). The warps sweep their
// rows once per pass of up to 8 columns: the products w_i v_i are formed once, in the
// first pass, and kept in shared memory, each lane reading back only what it wrote (no
// barrier inside a pass); a pass issues exactly its columns' FMAs, one per basis element
// read, two slabs of loads in flight per warp. A pass ends with one fold per warp (the 8
// partial sums halved across the lanes), a barrier, and a fixed-order sum over the 8
// warps; the block's sums go to partial[poff + j * nblk + blk]. The work of a job depends
// only on that job (its rows, k and nblk), so batched and separate launches give the
// same bits.
constexpr int kMaxCpw = 8;                       // columns per pass
constexpr int kWarpRows = 512;                   // rows per warp
constexpr int kBlockRows = kWarpRows * (kThreads / 32);

// Folds the 8 partial sums of every lane into warp totals: after the three halving steps
// (offsets 16, 8, 4) lane l holds a partial of column 4 bit4(l) + 2 bit3(l) + bit2(l),
// and two butterfly steps over lane bits 0-1 complete it. Fixed order: deterministic.
__device__ __forceinline__ double warp_fold8(double (&a)[kMaxCpw], int lane) {
  const unsigned full = 0xffffffffu;
  {
    const bool up = lane & 16;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double send = up ? a[q] : a[q + 4];
      const double keep = up ? a[q + 4] : a[q];
      a[q] = keep + __shfl_xor_sync(full, send, 16);
    }
  }
  {
    const bool up = lane & 8;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const double send = up ? a[q] : a[q + 2];
      const double keep = up ? a[q + 2] : a[q];
      a[q] = keep + __shfl_xor_sync(full, send, 8);
    }
  }
  {
    const bool up = lane & 4;
    const double send = up ? a[0] : a[1];
    const double keep = up ? a[1] : a[0];
    a[0] = keep + __shfl_xor_sync(full, send, 4);
  }
  double t = a[0];
  t += __shfl_xor_sync(full, t, 2);
  t += __shfl_xor_sync(full, t, 1);
  return t;
}
__device__ __forceinline__ int fold8_column(int lane) {
  return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// One pass of a warp over its rows for NC columns starting at Bc (column stride ldb).
// FIRST: form x_i = w_i v_i and keep it in xs (this lane's 16 slots); later passes read it.
template <int NC, bool FIRST>
__device__ __forceinline__ void mdot_pass(const DotJob& jb, const double* __restrict__ Bc, int64_t row0, int lane,
                                          double* xs, double (&acc)[kMaxCpw]) {
#pragma unroll 2
  for (int sl = 0; sl < kWarpRows / 32; ++sl) {
    const int64_t row = row0 + sl * 32 + lane;
    if (row < jb.n) {
      double x;
      if constexpr (FIRST) {
        x = jb.w ? jb.w[row] * jb.v[row] : jb.v[row];
        xs[sl * 32 + lane] = x;
      } else {
        x = xs[sl * 32 + lane];
      }
#pragma unroll
      for (int g = 0; g < NC; ++g) acc[g] = fma(__ldcs(Bc + g * jb.ldb + row), x, acc[g]);
    }
  }
}

template <bool FIRST>
__device__ __forceinline__ void mdot_pass_nc(int nc, const DotJob& jb, const double* __restrict__ Bc, int64_t row0,
                                             int lane, double* xs, double (&acc)[kMaxCpw]) {
  switch (nc) {
    case 8: mdot_pass<8, FIRST>(jb, Bc, row0, lane, xs, acc); break;
    case 7: mdot_pass<7, FIRST>(jb, Bc, row0, lane, xs, acc); break;
    case 6: mdot_pass<6, FIRST>(jb, Bc, row0, lane, xs, acc); break;
    case 5: mdot_pass<5, FIRST>(jb, Bc, row0, lane, xs, acc); break;
    case 4: mdot_pass<4, FIRST>(jb, Bc, row0, lane, xs, acc); break;
    case 3: mdot_pass<3, FIRST>(jb, Bc, row0, lane, xs, acc); break;
    case 2: mdot_pass<2, FIRST>(jb, Bc, row0, lane, xs, acc); break;
    default: mdot_pass<1, FIRST>(jb, Bc, row0, lane, xs, acc); break;
  }
}

__global__ void __launch_bounds__(kThreads, 4) k_mdot_jobs(const DotJob* __restrict__ jobs, int njobs,
                                                           double* __restrict__ partial) {
  __shared__ double s_x[kThreads / 32][kWarpRows];          // w_i v_i of each warp's rows
  __shared__ double s_red[kThreads / 32][kMaxCpw];
  const DotJob jb = jobs[job_of(jobs, njobs, blockIdx.x)];
  const int blk = static_cast<int>(blockIdx.x - jb.first);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = static_cast<int64_t>(blk) * kBlockRows + warp * kWarpRows;
  double* xs = s_x[warp];
  for (int c0 = 0; c0 < jb.k; c0 += kMaxCpw) {
    const int nc = min(kMaxCpw, jb.k - c0);
    const double* Bc = jb.B + static_cast<int64_t>(c0) * jb.ldb;
    double acc[kMaxCpw];
#pragma unroll
    for (int g = 0; g < kMaxCpw; ++g) acc[g] = 0.0;
    if (c0 == 0) mdot_pass_nc<true>(nc, jb, Bc, row0, lane, xs, acc);
    else mdot_pass_nc<false>(nc, jb, Bc, row0, lane, xs, acc);
    const double t = warp_fold8(acc, lane);
    const int g = fold8_column(lane);
    if ((lane & 3) == 0 && g < nc) s_red[warp][g] = t;
    __syncthreads();
    if (threadIdx.x < nc) {
      double sum = s_red[0][threadIdx.x];
#pragma unroll
      for (int wi = 1; wi < kThreads / 32; ++wi) sum += s_red[wi][threadIdx.x];
      partial[jb.poff + static_cast<int64_t>(c0 + threadIdx.x) * jb.nblk + blk] = sum;
    }
    __syncthreads();  // s_red is rewritten by the next pass
  }
}

__global__ void __launch_bounds__(kThreads) k_reduce_jobs(const DotJob* __restrict__ jobs,
                                                          const double* __restrict__ partial) {
  const DotJob jb = jobs[blockIdx.y];
  const int j = blockIdx.x;
  if (j >= jb.k) return;
  double v[1] = {0.0};
  for (int b = threadIdx.x; b < jb.nblk; b += kThreads) v[0] += partial[jb.poff + static_cast<int64_t>(j) * jb.nblk + b];
  double tot[1];
  block_sum<1>(v, tot);
  if (threadIdx.x == 0) jb.out[j] = tot[0];
}

__global__ void __launch_bounds__(kThreads) k_gemv_sub_jobs(const GemvJob* __restrict__ jobs, int njobs) {
  extern __shared__ double sh_h[];
  const GemvJob jb = jobs[job_of(jobs, njobs, blockIdx.x)];
  const int64_t blk = blockIdx.x - jb.first;
  for (int j = threadIdx.x; j < jb.k; j += kThreads) sh_h[j] = jb.h[j];
  __syncthreads();
  for (int64_t i = blk * static_cast<int64_t>(kThreads) + threadIdx.x; i < jb.n;
       i += static_cast<int64_t>(jb.nblk) * kThreads) {
    double s0 = 0.0, s1 = 0.0;
    int j = 0;
    for (; j + 2 <= jb.k; j += 2) {
      s0 = fma(jb.B[j * jb.ldb + i], sh_h[j], s0);
      s1 = fma(jb.B[(j + 1) * jb.ldb + i], sh_h[j + 1], s1);
    }
    if (j < jb.k) s0 = fma(jb.B[j * jb.ldb + i], sh_h[j], s0);
    jb.v[i] -= s0 + s1;
  }
}

// S x over every SELL slice, each mesh with its own vectors x_of[mesh] / y_of[mesh] (global
// row indexing; a null x_of skips the mesh's rows). Each row sum is one FMA chain from 0 in
// entry order, the sum the step kernels' SpMV forms, so it equals the per-mesh product.
__global__ void __launch_bounds__(kThreads) k_spmv_f64_meshes(SellDev A, const double* const* __restrict__ x_of,
                                                              double* const* __restrict__ y_of) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < A.n_slices;
       s += nwarps) {
    const int mesh = A.slice_mesh ? A.slice_mesh[s] : 0;
    const double* x = x_of[mesh];
    if (!x) continue;  // warp-uniform: a slice belongs to one mesh
    const int64_t beg = A.slice_ptr[s];
    const int w = static_cast<int>((A.slice_ptr[s + 1] - beg) >> 5);
    const double* v = A.val64 + beg + lane;
    const int32_t* c = A.col + beg + lane;
    double acc = 0.0;
    for (int k = 0; k < w; ++k) acc = fma(__ldcs(v + k * kSliceC), __ldg(x + __ldcs(c + k * kSliceC)), acc);
    y_of[mesh][s * kSliceC + lane] = acc;
  }
}

__global__ void k_scale_jobs(const ScaleJob* __restrict__ jobs) {
  const ScaleJob jb = jobs[blockIdx.y];
  const double nrm = sqrt(jb.nrm2[0]);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < jb.n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    jb.dst[i] = jb.v[i] / nrm;
}

}  // namespace

// Row blocks of a batched inner-product job: kBlockRows rows each.
int dot_blocks(int64_t n) {
  const int64_t b = (n + kBlockRows - 1) / kBlockRows;
  return static_cast<int>(b < 1 ? 1 : b);
}
int gemv_blocks(int64_t n) { return rows_grid(n, 2048); }

void launch_mdot_jobs(cudaStream_t st, const DotJob* jobs, int njobs, int max_k, int64_t total_blocks,
                      double* partial) {
  if (njobs <= 0 || max_k <= 0 || total_blocks <= 0) return;
  k_mdot_jobs<<<static_cast<unsigned>(total_blocks), kThreads, 0, st>>>(jobs, njobs, partial);
  k_reduce_jobs<<<dim3(max_k, njobs), kThreads, 0, st>>>(jobs, partial);
  g_launches += 2;
}

void launch_gemv_sub_jobs(cudaStream_t st, const GemvJob* jobs, int njobs, int max_k, int64_t total_blocks) {
  if (njobs <= 0 || max_k <= 0 || total_blocks <= 0) return;
  k_gemv_sub_jobs<<<static_cast<unsigned>(total_blocks), kThreads, max_k * sizeof(double), st>>>(jobs, njobs);
  ++g_launches;
}

void launch_spmv_f64_meshes(const SellDev& A, const LaunchCfg& cfg, cudaStream_t st, const double* const* x_of,
                            double* const* y_of) {
  const int64_t need = (A.n_slices + 7) / 8;  // 8 warps per block, a slice per warp
  const int64_t cap = static_cast<int64_t>(cfg.n_sm) * 8;
  k_spmv_f64_meshes<<<static_cast<int>(need < cap ? (need > 0 ? need : 1) : cap), kThreads, 0, st>>>(A, x_of, y_of);
  ++g_launches;
}

void launch_scale_jobs(cudaStream_t st, const ScaleJob* jobs, int njobs, int max_nblk) {
  if (njobs <= 0) return;
  k_scale_jobs<<<dim3(max_nblk, njobs), kThreads, 0, st>>>(jobs);
  ++g_launches;
}

void launch_mdot(cudaStream_t st, const double* B, int64_t ldb, int k, const double* v, const double* w,
                 int64_t n, double* partial, double* h) {
  if (k <= 0) return;
  const int nblk = rows_grid(n, kDotBlocks);
  dim3 grid(nblk, (k + kGroup - 1) / kGroup);
  k_mdot_partial<<<grid, kThreads, 0, st>>>(B, ldb, k, v, w, n, partial);
  k_reduce_partial<<<k, kThreads, 0, st>>>(partial, nblk, h);
  g_launches += 2;
}

void launch_gemv_sub(cudaStream_t st, double* v, const double* B, int64_t ldb, int k, const double* h,
                     int64_t n) {
  if (k <= 0) return;
  k_gemv_sub<<<rows_grid(n, 2048), kThreads, k * sizeof(double), st>>>(v, B, ldb, k, h, n);
  ++g_launches;
}

void launch_scale_rsqrt(cudaStream_t st, const double* v, const double* nrm2, double* dst, double* dst2,
                        int64_t n) {
  k_scale_rsqrt<<<rows_grid(n, 2048), kThreads, 0, st>>>(v, nrm2, dst, dst2, n);
  ++g_launches;
}

void launch_ritz_residual(cudaStream_t st, const double* B, const double* SB, int64_t ldb, int k,
                          const double* Y, const double* theta, int p, const double* m, int64_t n,
                          double* partial, double* out) {
  if (p <= 0) return;
  const int nblk = rows_grid(n, kDotBlocks);
  dim3 grid(nblk, (p + kGroup - 1) / kGroup);
  const size_t smem = static_cast<size_t>(k) * kGroup * sizeof(double);
  allow_dynamic_smem(reinterpret_cast<const void*>(&k_ritz_residual), smem);  // else the launch fails, reported
  k_ritz_residual<<<grid, kThreads, smem, st>>>(B, SB, ldb, k, Y, theta, p, m, n,
                                                                       partial);
  k_reduce_partial<<<2 * p, kThreads, 0, st>>>(partial, nblk, out);
  g_launches += 2;
}

void launch_gemm_bx(cudaStream_t st, const double* B, int64_t ldb, int k, const double* Y, int p, double* X,
                    int64_t ldx, int64_t n) {
  if (p <= 0) return;
  dim3 grid(rows_grid(n, 2048), (p + kGroup - 1) / kGroup);
  const size_t smem = static_cast<size_t>(k) * kGroup * sizeof(double);
  allow_dynamic_smem(reinterpret_cast<const void*>(&k_gemm_bx), smem);
  k_gemm_bx<<<grid, kThreads, smem, st>>>(B, ldb, k, Y, p, X, ldx, n);
  ++g_launches;
}

void launch_permute(cudaStream_t st, const double* src, double* dst, const int32_t* perm, int64_t n,
                    bool gather) {
  k_permute<<<rows_grid(n, 2048), kThreads, 0, st>>>(src, dst, perm, n, gather);
  ++g_launches;
}

void launch_scale(cudaStream_t st, const double* src, double s, double* dst, int64_t n) {
  k_scale<<<rows_grid(n, 2048), kThreads, 0, st>>>(src, s, dst, n);
  ++g_launches;
}

}  // namespace kes
