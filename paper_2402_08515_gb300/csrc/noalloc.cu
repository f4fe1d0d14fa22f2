// Allocation-free variant of the FP64 filter application.
//
// Some callers cannot call cudaMalloc at all: a host program that reserves
// every byte of device memory it may use when it starts and forbids any later
// allocation (a long-running service with a fixed memory budget, or a plugin
// whose host owns the device heap), so that a mid-run allocation can neither
// fail nor fragment memory. kes_create allocates its own state, so those
// callers get this entry point instead: they pass every input and the output
// in device memory they already own, and the two leapfrog state vectors live
// in the fixed array below, a file-scope __device__ array of this module.
//
// The array takes 2 * KES_NOALLOC_MAX_N doubles (16 MiB) on every device where
// this module is loaded, until the process exits. Under CUDA's default lazy
// module loading the module (and so the array) is loaded on a device by the
// first call there, when the set-up looks up the array's address: a caller that
// reserves all of its device memory must make one call first (or run with
// CUDA_MODULE_LOADING=EAGER, which loads every module with the context).
// Every call shares the array and it keeps the previous call's contents; calls
// whose GPU work overlaps (two streams, two host threads) race on it and must
// be serialised by the caller. Nothing has to start at zero: each call writes
// every state entry it reads.
#include <cuda_runtime.h>

#include <mutex>

#include "kes_internal.h"

static __device__ __align__(256) double kes_noalloc_state[2 * KES_NOALLOC_MAX_N];

namespace {

constexpr int kRowLanes = 8;   // lanes cooperating on one CSR row
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// One fused leapfrog step on CSR (the arithmetic of k_step_f64):
//   out = 2 x - prev - tau2m .* (S x);  acc = acc + alpha[step+1] * out
// first: prev = x and acc = alpha[0] * x + alpha[1] * out; last: out is not stored.
template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(kThreads) k_step_csr_f64(int64_t n, const int64_t* __restrict__ row_ptr,
                                                           const int32_t* __restrict__ col,
                                                           const double* __restrict__ val,
                                                           const double* __restrict__ tau2m,
                                                           const double* __restrict__ x, const double* prev,
                                                           double* out, double* acc,
                                                           const double* __restrict__ alpha, int step) {
  // kRowLanes lanes per row, 32 / kRowLanes rows per warp; the loop bound is uniform
  // across the warp so that every lane reaches the shuffles
  constexpr int kRowsPerWarp = 32 / kRowLanes;
  const int lane = threadIdx.x & 31;
  const int sub = lane % kRowLanes;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * kThreads) >> 5;
  for (int64_t base = warp * kRowsPerWarp; base < n; base += nwarps * kRowsPerWarp) {
    const int64_t row = base + lane / kRowLanes;
    double sum = 0.0;
    if (row < n)
      for (int64_t p = row_ptr[row] + sub; p < row_ptr[row + 1]; p += kRowLanes)
        sum = fma(val[p], __ldg(x + col[p]), sum);
#pragma unroll
    for (int o = kRowLanes / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, kRowLanes);
    if (sub == 0 && row < n) {
      const double xi = x[row];
      const double pi = FIRST ? xi : prev[row];
      const double un = fma(-tau2m[row], sum, 2.0 * xi - pi);
      if (!LAST) out[row] = un;
      acc[row] = fma(alpha[step + 1], un, FIRST ? alpha[0] * xi : acc[row]);
    }
  }
}

std::mutex g_setup_mu;
double* g_state[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t state_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_state[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, kes_noalloc_state);
    if (e != cudaSuccess) return e;
    g_state[dev] = static_cast<double*>(p);
  }
  *out = g_state[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" kes_status kes_filter_apply_noalloc(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                               const double* val, const double* tau2m, const double* alpha,
                                               int32_t L, const double* r_in, double* r_out, void* stream) {
  if (n < 1 || n > KES_NOALLOC_MAX_N || L < 1 || !row_ptr || !col || !val || !tau2m || !alpha || !r_in || !r_out)
    return KES_ERR_ARG;
  double* state = nullptr;
  if (state_for_current_device(&state) != cudaSuccess) {
    cudaGetLastError();
    return KES_ERR_CUDA;
  }
  double* U[2] = {state, state + KES_NOALLOC_MAX_N};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t want = (n * kRowLanes + kThreads - 1) / kThreads;  // one row group per 8 lanes
  const int grid = static_cast<int>(want < 4096 ? want : 4096);
  for (int s = 0; s < L; ++s) {
    const bool first = s == 0, last = s == L - 1;
    const double* x = s == 0 ? r_in : U[(s - 1) & 1];
    const double* prev = s <= 1 ? r_in : U[s & 1];
    double* out = U[s & 1];
    if (first && last)
      k_step_csr_f64<true, true><<<grid, kThreads, 0, st>>>(n, row_ptr, col, val, tau2m, x, prev, out, r_out, alpha, s);
    else if (first)
      k_step_csr_f64<true, false><<<grid, kThreads, 0, st>>>(n, row_ptr, col, val, tau2m, x, prev, out, r_out, alpha, s);
    else if (last)
      k_step_csr_f64<false, true><<<grid, kThreads, 0, st>>>(n, row_ptr, col, val, tau2m, x, prev, out, r_out, alpha, s);
    else
      k_step_csr_f64<false, false><<<grid, kThreads, 0, st>>>(n, row_ptr, col, val, tau2m, x, prev, out, r_out, alpha, s);
  }
  return cudaGetLastError() == cudaSuccess ? KES_OK : KES_ERR_CUDA;
}
