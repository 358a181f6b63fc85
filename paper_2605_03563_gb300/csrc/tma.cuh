// TMA (cp.async.bulk.tensor) and mbarrier helpers for the z-marching tile kernels.
//
// Tiles of a level array are staged plane by plane into shared memory by the
// Tensor Memory Accelerator: one elected thread arms an mbarrier with the
// byte count of a plane's boxes and issues the 3-D tile copies; every thread
// then waits on the barrier's phase.  Waits are bounded by the global timer:
// a copy that has not landed after kWaitNs sets the kernel's fault flag and the
// kernel runs to completion with whatever the buffer holds, so a fault is
// reported to the host instead of hanging the GPU.  Once a wait of the issuing
// thread has failed it issues no further copy; the copies already in flight
// (at most one per stage) are waited for, in order, up to kDrainNs each, so a
// CTA can only retire with a copy outstanding if that copy never completes.
#pragma once

#include <cuda.h>

#include "ps_common.cuh"

namespace ps {

static constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the async proxy (the TMA unit).
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier shared-memory accesses before later async-proxy writes.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the barrier phase with the given parity.  ok carries the kernel's
// state: while it is true a wait may take up to kWaitNs; once a wait has
// failed, later waits (which still drain the copies in flight, in order) give
// up after kDrainNs, so a faulty kernel ends within about kWaitNs.
static constexpr unsigned long long kDrainNs = 1000000ull;   // 1 ms
__device__ __forceinline__ void mbar_wait(unsigned long long* bar, unsigned parity, bool& ok) {
  if (mbar_try_wait(bar, parity)) return;
  const unsigned long long limit = ok ? kWaitNs : kDrainNs;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit) {
      ok = false;
      return;
    }
}

// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
// x * sizeof(element) must be a multiple of 16 bytes; y and z may be negative
// or past the end (those elements read as zero).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__host__ __device__ constexpr int align_up(int v, int a) { return (v + a - 1) / a * a; }

// Host: encode a tensor map over a level array of storage type dt (DType),
// logical extents (ex, ey, ez), row pitch px, box (bx, by, 1).  Returns false
// if the driver entry point is unavailable or the encoding is rejected.
bool encode_level_map(CUtensorMap* map, int dt, const void* base, const Dims& d, int bx, int by);

}  // namespace ps
