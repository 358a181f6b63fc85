// ps_probe_fp64: a throughput probe of the FP64 pipe.
//
// The FP64 kernels of the library (colour passes, FP64 residuals, multipole
// moments, the compact 27-point passes) are bound by the rate at which the
// GPU issues FP64 instructions, not by HBM.  Their roofline needs that rate
// measured on the device at hand, in the same process and at the same clocks
// as the kernel it is compared with.  This kernel issues nothing but FP64
// fused multiply-adds (kind 0) or FP64 adds (kind 1): every thread runs
// kChains independent dependency chains of `iters` instructions each, enough
// warps per SM to hide the pipe's latency, and writes one value per block so
// that no chain can be removed.
#include "ps_common.cuh"
#include "tma.cuh"

namespace ps {
namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_probe_fp64(int iters, double a, double b, double* out) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) {
      if (KIND == 0)
        asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[c]) : "d"(a), "d"(b));
      else
        asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(x[c]) : "d"(b));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  __shared__ double sh[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; w++) t += sh[w];
    out[blockIdx.x] = t;
  }
}

// One warp waits on an mbarrier that nothing ever arrives at, through the same
// bounded wait the TMA tile kernels use (the first wait of a kernel, or a wait
// after an earlier one has failed), then reports whether it gave up and how
// long it waited.
__global__ void k_probe_bounded_wait(int first_wait, long long* out) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  bool ok = first_wait != 0;
  const unsigned long long t0 = global_ns();
  mbar_wait(&bar, 0, ok);
  const unsigned long long t1 = global_ns();
  const bool phase_done = mbar_try_wait(&bar, 0);
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = phase_done ? 0 : 1;          // 1: the wait gave up (the phase never completed)
    out[1] = (long long)(t1 - t0);
    out[2] = ok ? 0 : 1;                  // the kernel's fault state after the wait
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
  }
}

}  // namespace
}  // namespace ps

using namespace ps;

extern "C" ps_status ps_probe_bounded_wait(int first_wait, long long* out_dev, double* waited_ms_host,
                                           void* stream) {
  if (out_dev == nullptr) {
    set_error("ps_probe_bounded_wait: out_dev must be non-NULL");
    return PS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_probe_bounded_wait<<<1, 32, 0, s>>>(first_wait != 0 ? 1 : 0, out_dev);
  long long h[3] = {0, 0, 0};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, out_dev, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error("ps_probe_bounded_wait: %s", cudaGetErrorString(e));
    return PS_ERR_CUDA;
  }
  if (waited_ms_host) *waited_ms_host = (double)h[1] * 1e-6;
  if (h[0] != 0 && h[2] != 0) {
    set_error("ps_probe_bounded_wait: the bounded wait ran out after %.3f ms", (double)h[1] * 1e-6);
    return PS_ERR_TIMEOUT;
  }
  if (h[0] != 0) {
    set_error("ps_probe_bounded_wait: the wait returned without its phase and without a fault");
    return PS_ERR_CUDA;
  }
  return PS_OK;
}

extern "C" ps_status ps_probe_fp64(int kind, int blocks, int iters, double* out_dev,
                                   double* instructions_host, void* stream) {
  if ((kind != 0 && kind != 1) || blocks < 1 || blocks > (1 << 20) || iters < 1 || iters > (1 << 24) ||
      out_dev == nullptr) {
    set_error("ps_probe_fp64: kind must be 0 or 1, 1 <= blocks <= 2^20, 1 <= iters <= 2^24, out_dev non-NULL");
    return PS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a = 1 - 2^-20 and b = 2^-20 keep every chain near 1 (no overflow, no denormals)
  const double a = 1.0 - 9.5367431640625e-07, b = 9.5367431640625e-07;
  if (kind == 0)
    k_probe_fp64<0><<<blocks, kThreads, 0, s>>>(iters, a, b, out_dev);
  else
    k_probe_fp64<1><<<blocks, kThreads, 0, s>>>(iters, a, b, out_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("ps_probe_fp64: launch failed: %s", cudaGetErrorString(e));
    return PS_ERR_CUDA;
  }
  if (instructions_host) *instructions_host = (double)blocks * kThreads * kChains * (double)iters;
  return PS_OK;
}
