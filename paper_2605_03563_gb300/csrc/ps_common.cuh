// Common device/host helpers of the GB300 Poisson library.
//
// Storage types: double, float, __nv_bfloat16.  Arithmetic type: double for
// double storage, float otherwise.  Reductions always accumulate in double and
// are deterministic: a fixed xor-shuffle tree per warp, a fixed tree per block,
// per-block partials summed in block order by a single-block finisher.
#pragma once
#include <climits>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/poisson.h"

namespace ps {

// ------------------------------------------------------------ storage traits
template <typename T> struct St;
template <> struct St<double> {
  using C = double;
  static __device__ __forceinline__ double ld(const double* p) { return *p; }
  static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
};
template <> struct St<float> {
  using C = float;
  static __device__ __forceinline__ float ld(const float* p) { return *p; }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <> struct St<__nv_bfloat16> {
  using C = float;
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// Two adjacent values stored with one vector store (p aligned to the pair), and
// the value a store of type T keeps (rounding to BF16 where T is BF16).
template <typename T> struct St2;
template <> struct St2<double> {
  static __device__ __forceinline__ void st(double* p, double a, double b) {
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
  }
};
template <> struct St2<float> {
  static __device__ __forceinline__ void st(float* p, float a, float b) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
  }
};
template <> struct St2<__nv_bfloat16> {
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
  }
};
template <typename T> __device__ __forceinline__ typename St<T>::C stored(typename St<T>::C v) { return v; }
template <> __device__ __forceinline__ float stored<__nv_bfloat16>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

// ------------------------------------------------------------ Cartesian level geometry
// Logical extents (ex,ey,ez) = n + 2g - 1 per axis, x fastest; node index i sits at
// array index i + g - 1; interior unknowns occupy array indices [g, n + g - 2].
// Rows are px >= ex elements apart: caller-owned arrays are dense (px = ex);
// the library's own level arrays pad rows to a multiple of 32 elements so that
// every row starts on a 16-byte boundary (TMA tensor maps need 16-byte strides).
struct Dims {
  int nx, ny, nz;   // intervals
  int g;            // stencil radius (ghost width)
  int ex, ey, ez;   // logical array extents
  int px;           // row pitch in elements
  __host__ __device__ long long size() const { return (long long)px * ey * ez; }
  __host__ __device__ long long at(int i, int j, int k) const {
    return ((long long)k * ey + j) * px + i;
  }
  __host__ __device__ long long sy() const { return px; }
  __host__ __device__ long long sz() const { return (long long)px * ey; }
  __host__ __device__ int ni() const { return nx - 1; }   // interior counts
  __host__ __device__ int nj() const { return ny - 1; }
  __host__ __device__ int nk() const { return nz - 1; }
};

inline Dims make_dims(int nx, int ny, int nz, int g, int align = 1) {
  Dims d;
  d.nx = nx; d.ny = ny; d.nz = nz; d.g = g;
  d.ex = nx + 2 * g - 1; d.ey = ny + 2 * g - 1; d.ez = nz + 2 * g - 1;
  d.px = (d.ex + align - 1) / align * align;
  return d;
}

// Scaled stencil coefficients.  With d = -(diagonal of A) > 0 the Gauss-Seidel
// value of a node is  phi_GS = sum_a c1[a](phi_{+1}+phi_{-1}) + c2[a](phi_{+2}+phi_{-2}) + fs
// where fs = -f/d is the scaled right-hand side; delta = phi_GS - phi and the
// residual is r = f - A phi = -d * delta.
template <typename C> struct Coef {
  C c1[3];
  C c2[3];
  double d;          // -(diagonal), kept in double for norms
  double inv_d;
};

// ------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Nodes per thread of the FP64 diagonal walks of a level with nk interior
// planes.  Any length gives the same values; shorter walks run more threads
// (latency hiding on the smaller levels) and start afresh more often (one
// more FP64 add per walk).  Measured on the 256^3 FP64 solve: 16 / 8 / 4
// nodes (>= 200 / >= 64 / below) 12.68 ms, the lengths below 12.34 ms.
inline int diag_walk_len(int nk) {
  return nk >= 400 ? 16 : (nk >= 200 ? 8 : (nk >= 100 ? 4 : (nk >= 24 ? 2 : 1)));
}

// Running max |x| of FP64 values without FP64 instructions: non-negative
// doubles order like their bit patterns, compared here as (high word, low
// word) pairs of 32-bit integers (a 64-bit integer max issues at about the
// FP64 rate on this part; the 32-bit compares and selects do not).
struct AbsMax {
  unsigned hi = 0u, lo = 0u;
  __device__ __forceinline__ void take(double v) {
    const unsigned h = (unsigned)__double2hiint(v) & 0x7fffffffu, l = (unsigned)__double2loint(v);
    take_bits(h, l);
  }
  __device__ __forceinline__ void take_bits(unsigned h, unsigned l) {
    const bool gt = h > hi || (h == hi && l > lo);
    hi = gt ? h : hi;
    lo = gt ? l : lo;
  }
  __device__ __forceinline__ double value() const { return __hiloint2double((int)hi, (int)lo); }
};

// Max over the warp of |v| (the bit order of AbsMax, integer pipe only).
__device__ __forceinline__ double warp_absmax(double v) {
  AbsMax a;
  a.take(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    a.take_bits(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
  return a.value();
}

// Block-wide sum of NV values per thread, result valid in thread 0.
// `sh` must hold 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int lane = tid & 31, warp = tid >> 5, nw = (nthr + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; q++) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) sh[q * 32 + warp] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) {
      double x = lane < nw ? sh[q * 32 + lane] : 0.0;
      v[q] = warp_sum(x);
    }
  }
}

// 1/p for p = 2^e, |e| <= 1022, by negating the exponent field (an integer
// subtraction; no FP64 division); other p divide.
__device__ __forceinline__ double inverse_scale(double p) {
  const long long b = __double_as_longlong(p);
  const long long e = (b >> 52) & 0x7ff;
  if ((b & 0x000fffffffffffffLL) == 0 && b > 0 && e >= 1 && e <= 2045)
    return __longlong_as_double(0x7fe0000000000000LL - b);
  return 1.0 / p;
}

// Exponent e of p when p = 2^e exactly with |e| <= 100, else INT_MIN.
__device__ __forceinline__ int pow2_exponent(double p) {
  const long long b = __double_as_longlong(p);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  return ((b & 0x000fffffffffffffLL) == 0 && b > 0 && e >= -100 && e <= 100) ? e : INT_MIN;
}

// x * 2^e rounded to the nearest binary32 (ties to even), for finite x and
// |e| <= 100, computed on the integer pipe from the binary64 encoding
// (IEEE 754 round-to-nearest-even applied to the 53-bit significand):
//   result exponent fe = ex - 1023 + 127 + e; normal results keep the top 23
//   fraction bits and round on the 29 dropped ones; results below the binary32
//   normal range shift the significand (implicit bit included) right by
//   29 + 1 - fe; a carry out of the fraction moves into the exponent, which
//   also yields the smallest normal and infinity where they are the rounded
//   values.  It replaces a conversion instruction of the FP64 pipe.
__device__ __forceinline__ float f64_to_f32_pow2(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return __uint_as_float(sign);   // zero, or below 2^-1022 (2^-922 after scaling): rounds to 0
  const int fe = ex - 1023 + 127 + e;
  if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned long long frac = b & 0x000fffffffffffffull;
  if (fe >= 1) {
    const unsigned m = (unsigned)(frac >> 29);
    const unsigned rest = (unsigned)frac & 0x1fffffffu;
    unsigned r = ((unsigned)fe << 23) | m;
    if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) r += 1u;
    return __uint_as_float(sign | r);
  }
  const int sh = 30 - fe;   // >= 30
  if (sh > 54) return __uint_as_float(sign);   // below half the smallest subnormal
  const unsigned long long sig = frac | 0x0010000000000000ull;
  unsigned q = (unsigned)(sig >> sh);
  const unsigned long long rest = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  if (rest > half || (rest == half && (q & 1u))) q += 1u;
  return __uint_as_float(sign | q);
}

// v * 2^e as binary64 for a binary32 v and |e| <= 100, built from v's encoding
// on the integer pipe: the product is exact in binary64 (its exponent range
// covers 2^(-149-100) .. 2^(128+100)), so only the exponent moves; binary32
// subnormals are normalised with a count of leading zeros; zeros, infinities
// and NaNs keep their class.  It replaces the FP64 pipe's conversion and
// multiply (a DADD of the result rounds exactly as an FMA of v, 2^e and the
// addend would).
__device__ __forceinline__ double f32_to_f64_pow2(float v, int e) {
  const unsigned b = __float_as_uint(v);
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const int ex = (int)((b >> 23) & 0xffu);
  unsigned frac = b & 0x7fffffu;
  if (ex == 0xff)   // infinity or NaN
    return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | ((unsigned long long)frac << 29)));
  int E;
  if (ex == 0) {
    if (frac == 0u) return __longlong_as_double((long long)sign);
    const int p = 31 - __clz(frac);   // leading bit: value = 1.f x 2^(p - 149)
    E = p - 149;
    frac = (frac << (23 - p)) & 0x7fffffu;
  } else {
    E = ex - 127;
  }
  const unsigned long long bits =
      sign | ((unsigned long long)(E + e + 1023) << 52) | ((unsigned long long)frac << 29);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ int block_linear_id() {
  return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// ------------------------------------------------------------ device solver state
// One per solve; lives in device memory, copied to pinned host memory for
// progress checks.  Kernels of an iteration body skip their work once done != 0.
struct DevState {
  double ref;         // reference norm (denominator of the relative residual)
  double rr;          // latest squared residual norm (unscaled)
  double rel;         // latest relative residual
  double rel0;        // initial relative residual
  double tol;
  double amax;        // max |delta| of the latest residual pass
  double scale_cur;   // IR: power-of-two scale of the inner RHS being solved
  double scale_next;  // IR: scale the next stored inner RHS will use
  // Krylov scalars
  double alpha, beta, omega, rho, rho_new, pq, ts, tt, ss;
  int iter;
  int max_iter;
  int done;           // 1 converged, 2 not converged (max_iter), 3 diverged
  int coarse_iter_last;
  int chunk_end;      // a captured loop continues while iter < chunk_end (set per step)
  int guess_nonzero;  // set-up copy: some interior node of the initial guess is nonzero
  long long coarse_iter_total;
  long long inner_cycles;   // IR inner cycles; FP32 BiCGSTAB: residual replacements
  // BiCGSTAB: breakdown restart and residual replacement
  double rmax;        // largest recurrence residual norm since the last replacement
  int broke;          // alpha or omega broke down in this iteration
  int restart;        // the next direction update restarts rhat = p = r
  int replace;        // the true residual replaces the recurrence one this iteration
  int fault;          // a tile kernel's TMA copy did not complete in time
  double replace_drop;     // BiCGSTAB: replace when ||r|| <= replace_drop * rmax
  int restart_on_replace;  // BiCGSTAB: restart rhat = p = r at every replacement
  int iter_repl;           // BiCGSTAB: iteration of the last replacement
  int discard;             // refinement form: the inner solve failed, drop its increments
  int inner_cap;           // refinement form: most iterations of the current inner solve
  int lag_pending;         // lagged-norm V-cycles: a first colour pass with saved values ran this step
};

enum { DONE_NO = 0, DONE_CONVERGED = 1, DONE_MAXITER = 2, DONE_DIVERGED = 3, DONE_FAULT = 4 };

}  // namespace ps

#define PS_CUDA_TRY(expr)                                                     \
  do {                                                                        \
    cudaError_t _e = (expr);                                                  \
    if (_e != cudaSuccess) {                                                  \
      ps::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr,               \
                    cudaGetErrorString(_e));                                  \
      return PS_ERR_CUDA;                                                     \
    }                                                                         \
  } while (0)

namespace ps {
void set_error(const char* fmt, ...);
// Streaming multiprocessors of the current device (queried once per device and
// cached); launch geometries scale with it.
int device_sm_count();
}
