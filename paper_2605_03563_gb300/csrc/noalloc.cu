// ps_op_residual_noalloc: the residual r = f - A phi and ||r||^2 on FP64
// Cartesian fields, computed without allocating any device memory.
//
// Who needs this: callers that are not allowed to call cudaMalloc themselves
// or through us -- for example code running inside a memory pool or arena
// that owns every allocation on the device, real-time loops where a device
// allocation could stall or fail, or hosts embedding the library under a
// no-allocation policy.  ps_op_residual allocates two temporary buffers per
// call; this variant instead keeps its scratch (the per-block partial sums of
// r^2 and the final sum) in one fixed array in device global memory that is
// part of the loaded library.
//
// Limits and sharing rules:
//  * the scratch holds kMaxSlots per-block partials: grids whose launch needs
//    more blocks (more than 32768, i.e. beyond about 512^3 intervals) are
//    rejected with PS_ERR_INVALID_ARG before any GPU work;
//  * every GPU that loads the library keeps this array (256 KB) until exit;
//  * all calls on a device share the one array and it keeps the last call's
//    contents, so calls whose kernels may overlap on the GPU (different
//    streams, or threads sharing a device) race on it: serialise them;
//  * every slot a call reads is written earlier in the same call, so nothing
//    has to be cleared between calls;
//  * the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture.  The address is cached for the life of the
//    process, so it goes stale if the device's primary context is torn down
//    (cudaDeviceReset): the entry point must not be called on that device
//    again afterwards.
#include <mutex>

#include "cart_kernels.cuh"

namespace ps {
namespace {

constexpr int kMaxSlots = 32768;
constexpr int kResultSlot = kMaxSlots;
constexpr int NB_X = 32, NB_Y = 8, NB_Z = 16;

// The scratch.  Host code must not pass this name to a kernel (on the host it
// is only a stand-in for the symbol); it uses the address looked up below.
static __device__ __align__(256) double g_noalloc_scratch[kMaxSlots + 32];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// r = f - A phi on interior nodes, one partial sum of r^2 per block.
template <int G>
__global__ void __launch_bounds__(NB_X* NB_Y)
    k_residual_noalloc(Dims d, double cx, double cy, double cz, double w0, double w1, double w2,
                       const double* __restrict__ phi, const double* __restrict__ f,
                       double* __restrict__ r, double* __restrict__ partials) {
  __shared__ double sh[32];
  const int i = blockIdx.x * NB_X + threadIdx.x + G;
  const int j = blockIdx.y * NB_Y + threadIdx.y + G;
  const int k0 = blockIdx.z * NB_Z + G, k1 = min(k0 + NB_Z, G + d.nk());
  const long long sy = d.sy(), sz = d.sz();
  double s2 = 0.0;
  if (i < G + d.ni() && j < G + d.nj()) {
    for (int k = k0; k < k1; k++) {
      const long long p = d.at(i, j, k);
      const double c = phi[p];
      double ax = w1 * (phi[p + 1] + phi[p - 1]) + w0 * c;
      double ay = w1 * (phi[p + sy] + phi[p - sy]) + w0 * c;
      double az = w1 * (phi[p + sz] + phi[p - sz]) + w0 * c;
      if (G == 2) {
        ax += w2 * (phi[p + 2] + phi[p - 2]);
        ay += w2 * (phi[p + 2 * sy] + phi[p - 2 * sy]);
        az += w2 * (phi[p + 2 * sz] + phi[p - 2 * sz]);
      }
      const double rv = f[p] - (cx * ax + cy * ay + cz * az);
      r[p] = rv;
      s2 = fma(rv, rv, s2);
    }
  }
  double v[1] = {s2};
  block_sum<1>(v, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) partials[block_linear_id()] = v[0];
}

// Sum the partials in block order into the result slot.
__global__ void k_sum_noalloc(const double* __restrict__ partials, int n, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) s += partials[b];
  double v[1] = {s};
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) *out = v[0];
}

}  // namespace
}  // namespace ps

using namespace ps;

extern "C" ps_status ps_op_residual_noalloc(const ps_grid* grid, int stencil_order,
                                            const double* phi, const double* f, double* r,
                                            double* norm2_host, void* stream) {
  if (!grid || grid->kind != PS_GRID_CART_UNIFORM) {
    set_error("ps_op_residual_noalloc: Cartesian grid required");
    return PS_ERR_INVALID_ARG;
  }
  if (stencil_order != 2 && stencil_order != 4) {
    set_error("ps_op_residual_noalloc: stencil_order must be 2 or 4 (got %d)", stencil_order);
    return PS_ERR_INVALID_ARG;
  }
  for (int a = 0; a < 3; a++) {
    if (grid->n[a] < 2 || grid->n[a] > 8192 || !(grid->hi[a] > grid->lo[a])) {
      set_error("ps_op_residual_noalloc: bad extent on axis %d", a);
      return PS_ERR_INVALID_ARG;
    }
  }
  if (!phi || !f || !r) {
    set_error("ps_op_residual_noalloc: NULL buffer");
    return PS_ERR_INVALID_ARG;
  }
  const Dims d = make_dims(grid->n[0], grid->n[1], grid->n[2], stencil_order / 2);
  const dim3 blocks((d.ni() + NB_X - 1) / NB_X, (d.nj() + NB_Y - 1) / NB_Y, (d.nk() + NB_Z - 1) / NB_Z);
  const long long nblocks = (long long)blocks.x * blocks.y * blocks.z;
  if (nblocks > kMaxSlots) {
    set_error("ps_op_residual_noalloc: grid %dx%dx%d needs %lld reduction slots; the fixed scratch "
              "holds %d (use ps_op_residual for larger grids)",
              grid->n[0], grid->n[1], grid->n[2], nblocks, kMaxSlots);
    return PS_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    set_error("ps_op_residual_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    return PS_ERR_CUDA;
  }
  double ih2[3];
  for (int a = 0; a < 3; a++) {
    const double h = (grid->hi[a] - grid->lo[a]) / grid->n[a];
    ih2[a] = 1.0 / (h * h);
  }
  const double w0 = stencil_order == 2 ? -2.0 : -30.0 / 12.0;
  const double w1 = stencil_order == 2 ? 1.0 : 16.0 / 12.0;
  const double w2 = stencil_order == 2 ? 0.0 : -1.0 / 12.0;
  cudaStream_t s = (cudaStream_t)stream;
  if (stencil_order == 2)
    k_residual_noalloc<1><<<blocks, dim3(NB_X, NB_Y), 0, s>>>(d, ih2[0], ih2[1], ih2[2], w0, w1, w2, phi, f, r, scratch);
  else
    k_residual_noalloc<2><<<blocks, dim3(NB_X, NB_Y), 0, s>>>(d, ih2[0], ih2[1], ih2[2], w0, w1, w2, phi, f, r, scratch);
  k_sum_noalloc<<<1, 256, 0, s>>>(scratch, (int)nblocks, scratch + kResultSlot);
  e = cudaGetLastError();
  if (e == cudaSuccess && norm2_host != nullptr) {
    e = cudaMemcpyAsync(norm2_host, scratch + kResultSlot, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) {
    set_error("ps_op_residual_noalloc: %s", cudaGetErrorString(e));
    return PS_ERR_CUDA;
  }
  return PS_OK;
}
