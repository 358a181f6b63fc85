// Cartesian stencil kernels of the GB300 Poisson library.
//
// Operators (Eq. 1 on a vertex-centred uniform grid, Sec. 2.1):
//   order 2: 7-point   sum_a (phi_{+1} - 2 phi + phi_{-1}) / h_a^2
//   order 4: 13-point  sum_a (-phi_{+2} + 16 phi_{+1} - 30 phi + 16 phi_{-1} - phi_{-2}) / (12 h_a^2)
// Every kernel works in the scaled Gauss-Seidel form: with d = -(diagonal) the
// GS value is  phi_GS = sum_a c1_a (phi_{+-1}) + c2_a (phi_{+-2}) + fs,  fs = -f/d,
// and delta = phi_GS - phi = -(f - A phi)/d.  This needs the fewest FP64
// instructions per node (6 for an isotropic 7-point GS update), which matters
// because the GB300 FP64 pipe issues ~0.6 T instructions/s while HBM delivers
// ~6.6 TB/s: FP64 sweeps are bound by FP64 issue, FP32/BF16 sweeps by HBM.
//
// Launch geometry of the point kernels: 32 x 8 threads per block over (x, y)
// and a z-chunk of nodes per thread chosen per level (zchunk_for): deep chunks
// on the large finest levels, one node per thread on small levels so that the
// launch still fills every SM instead of serialising memory latency along z.
// Kernels recover the chunk from gridDim.z.
#include <algorithm>
#include <cstdio>

#include "cart_kernels.cuh"
#include "stencil.cuh"

namespace ps {

static constexpr int BX = 32, BY = 8, ZCH = 16;
static inline int zchunk_for(int gxy, int nk) {
  // about 8 blocks per SM
  long long z = (long long)gxy * nk / (8LL * device_sm_count());
  return (int)std::max(1LL, std::min((long long)ZCH, z));
}

// z-chunk of the current launch
__device__ __forceinline__ int zchunk(int nk) { return (nk + gridDim.z - 1) / gridDim.z; }

template <typename C>
Coef<C> make_coef(const Dims& d, const double h[3], int order) {
  (void)d;
  Coef<C> cf;
  double w0 = order == 2 ? -2.0 : -30.0 / 12.0;
  double w1 = order == 2 ? 1.0 : 16.0 / 12.0;
  double w2 = order == 2 ? 0.0 : -1.0 / 12.0;
  double ih2[3], sum = 0.0;
  for (int a = 0; a < 3; a++) { ih2[a] = 1.0 / (h[a] * h[a]); sum += ih2[a]; }
  double dd = -w0 * sum;
  for (int a = 0; a < 3; a++) {
    cf.c1[a] = (C)(w1 * ih2[a] / dd);
    cf.c2[a] = (C)(w2 * ih2[a] / dd);
  }
  cf.d = dd;
  cf.inv_d = 1.0 / dd;
  return cf;
}
template Coef<double> make_coef<double>(const Dims&, const double*, int);
template Coef<float> make_coef<float>(const Dims&, const double*, int);

static inline bool is_iso(const double h[3]) { return h[0] == h[1] && h[1] == h[2]; }

static inline dim3 point_grid(const Dims& d) {
  const int gx = (d.ni() + BX - 1) / BX, gy = (d.nj() + BY - 1) / BY;
  const int zc = zchunk_for(gx * gy, d.nk());
  return dim3(gx, gy, (d.nk() + zc - 1) / zc);
}

int cart_partials_count(const Dims& d) {
  const dim3 g = point_grid(d);
  return g.x * g.y * g.z;
}

// Same with every interior neighbour read as zero (reference norm only).
template <int G, typename T, typename C>
__device__ __forceinline__ C gs_value_zero_interior(const T* __restrict__ phi, const Dims& d, int i, int j, int k,
                                    const Coef<C>& cf, C fs) {
  using S = St<T>;
  // every neighbour interior (all but the nodes next to the boundary): the
  // neighbour terms vanish; fs is returned as it is (fs + 0 differs from it
  // only in the sign of a zero, which neither the square nor the magnitude
  // the reference norm takes can see)
  if (i >= 2 * G && i < d.ni() && j >= 2 * G && j < d.nj() && k >= 2 * G && k < d.nk()) return fs;
  auto val = [&](int ii, int jj, int kk) -> C {
    bool inside = ii >= G && ii < G + d.ni() && jj >= G && jj < G + d.nj() && kk >= G &&
                  kk < G + d.nk();
    return inside ? (C)0 : S::ld(phi + d.at(ii, jj, kk));
  };
  C v = fs;
  for (int o = 1; o <= G; o++) {
    C ax = val(i + o, j, k) + val(i - o, j, k);
    C ay = val(i, j + o, k) + val(i, j - o, k);
    C az = val(i, j, k + o) + val(i, j, k - o);
    const C* c = o == 1 ? cf.c1 : cf.c2;
    v += ax * c[0] + ay * c[1] + az * c[2];
  }
  return v;
}

template <typename T>
__device__ __forceinline__ void store_dt(void* out, int dt, long long p, double v) {
  if (dt == DT_F64) ((double*)out)[p] = v;
  else if (dt == DT_F32) ((float*)out)[p] = (float)v;
  else ((__nv_bfloat16*)out)[p] = __float2bfloat16_rn((float)v);
}

// Block reduction of {sum, max} into partials[2*block], partials[2*block+1];
// m >= 0 (a max of magnitudes), reduced by its bits on the integer pipe.
__device__ __forceinline__ void block_sum_max(double s, double m, double* partials) {
  __shared__ double sh[64];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
  s = warp_sum(s);
  m = warp_absmax(m);
  if (lane == 0) { sh[warp] = s; sh[32 + warp] = m; }
  __syncthreads();
  if (warp == 0) {
    double a = lane < nw ? sh[lane] : 0.0;
    double b = lane < nw ? sh[32 + lane] : 0.0;
    a = warp_sum(a);
    b = warp_absmax(b);
    if (lane == 0) {
      int bid = block_linear_id();
      partials[2 * bid] = a;
      partials[2 * bid + 1] = b;
    }
  }
}

// Block {sum, max} of FP32 per-thread values of a scaled quantity x * scale:
// warps reduce in FP32 (the per-thread sums already are FP32), each warp's
// result is unscaled once in FP64 and the warps are combined in FP64, so the
// FP64 pipe sees a few instructions per warp instead of per thread.
__device__ __forceinline__ void block_sum_max_scaled(float s, float m, double scale, double* partials) {
  __shared__ double sh[64];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if (lane == 0) {
    const double inv = inverse_scale(scale);
    sh[warp] = (double)s * inv * inv;
    sh[32 + warp] = (double)m * inv;
  }
  __syncthreads();
  if (warp == 0) {
    double a = lane < nw ? sh[lane] : 0.0;
    double b = lane < nw ? sh[32 + lane] : 0.0;
    a = warp_sum(a);
    b = warp_max(b);
    if (lane == 0) {
      int bid = block_linear_id();
      partials[2 * bid] = a;
      partials[2 * bid + 1] = b;
    }
  }
}

// ------------------------------------------------------------------ delta pass
// RED: 0 no reduction, 1 sum of delta^2, 2 sum of delta^2 and max |delta|.
template <int G, bool ISO, typename TI, int RED>
__global__ void __launch_bounds__(BX* BY)
    k_delta(Dims d, Coef<typename St<TI>::C> cf, const TI* __restrict__ phi,
            const TI* __restrict__ fs, int dout, void* __restrict__ out, double out_scale,
            const DevState* __restrict__ st, int zero_interior, double* __restrict__ partials) {
  using C = typename St<TI>::C;
  using S = St<TI>;
  const int i = blockIdx.x * BX + threadIdx.x + G;
  const int j = blockIdx.y * BY + threadIdx.y + G;
  const int zc = zchunk(d.nk());
  const int k0 = blockIdx.z * zc + G;
  const int k1 = min(k0 + zc, G + d.nk());
  const long long sy = d.sy(), sz = d.sz();
  double s2 = 0.0, mx = 0.0;
  AbsMax mxb;   // max |delta| without FP64 instructions
  float s2f = 0.0f, mxf = 0.0f;
  double oscale = out_scale;
  if (st != nullptr) oscale = st->scale_next;
  // a power-of-two scale 2^e (|e| <= 100) is applied inside the integer-pipe conversion
  const int oexp = pow2_exponent(oscale);
  if (i < G + d.ni() && j < G + d.nj()) {
    // two z nodes per trip: their loads and FP64 chains are independent
#pragma unroll 2
    for (int k = k0; k < k1; k++) {
      const long long p = d.at(i, j, k);
      C dl;
      if (zero_interior) {
        dl = gs_value_zero_interior<G>(phi, d, i, j, k, cf, S::ld(fs + p));
      } else {
        dl = gs_value<G, ISO>(phi, p, sy, sz, cf, S::ld(fs + p)) - S::ld(phi + p);
      }
      const double dd = (RED >= 1 || sizeof(C) == sizeof(double)) ? (double)dl : 0.0;
      if (RED == 2 && dout != DT_F64) {
        // refinement pass: the stored inner right-hand side is FP32/BF16, so the
        // sum of squares and the max run on the FP32 pipe over the scaled value
        // (O(1) by the choice of the power-of-two scale; exact to undo).  The
        // scaled value is rounded to FP32 on the integer pipe (no FP64 conversion
        // or multiply).
        const float v = oexp != INT_MIN ? f64_to_f32_pow2(dd, oexp) : (float)(dd * oscale);
        s2f = fmaf(v, v, s2f);
        mxf = fmaxf(mxf, fabsf(v));
        if (dout == DT_F32) ((float*)out)[p] = v;
        else ((__nv_bfloat16*)out)[p] = __float2bfloat16_rn(v);
        continue;
      }
      if (RED >= 1) s2 = fma(dd, dd, s2);
      if (RED == 2) mxb.take(dd);
      if (out != nullptr) {
        if (sizeof(C) == sizeof(float)) {
          // FP32 arithmetic levels never touch the FP64 pipe on the store path
          const float v = (float)dl * (float)oscale;
          if (dout == DT_F32) ((float*)out)[p] = v;
          else if (dout == DT_BF16) ((__nv_bfloat16*)out)[p] = __float2bfloat16_rn(v);
          else ((double*)out)[p] = (double)v;
        } else {
          store_dt<C>(out, dout, p, dd * oscale);
        }
      }
    }
  }
  if (RED == 2 && dout != DT_F64) {
    block_sum_max_scaled(s2f, mxf, oscale, partials);
    return;
  }
  if (RED == 2) mx = mxb.value();
  if (RED >= 1) block_sum_max(s2, mx, partials);
}

// Set-up copy of the caller's initial guess (dense rows) into the handle's
// pitched array, one warp per row.  It records in st->guess_nonzero whether
// any interior node of the guess is nonzero (+0 and -0 both count as zero):
// from a zero guess the initial residual f - A phi0 is the reference vector,
// and the initial residual pass takes the reference norm instead.
__global__ void __launch_bounds__(256)
    k_copy_guess(Dims dd, Dims sd, const double* __restrict__ src, double* __restrict__ dst,
                 DevState* __restrict__ st) {
  const long long rows = (long long)sd.ey * sd.ez;
  const long long row = blockIdx.x * 8LL + (threadIdx.x >> 5);
  int nz = 0;
  if (row < rows) {
    const int j = (int)(row % sd.ey), k = (int)(row / sd.ey), g = sd.g;
    const bool inrow = j >= g && j < sd.ey - g && k >= g && k < sd.ez - g;
    const double* a = src + row * sd.px;
    double* b = dst + row * dd.px;
#pragma unroll 4
    for (int i = threadIdx.x & 31; i < sd.ex; i += 32) {
      const double v = a[i];
      b[i] = v;
      if (inrow && i >= g && i < sd.ex - g && ((unsigned long long)__double_as_longlong(v) << 1) != 0ull) nz = 1;
    }
  }
  if (__syncthreads_or(nz) && threadIdx.x == 0) st->guess_nonzero = 1;
}

cudaError_t launch_copy_guess(const Dims& dd, const Dims& sd, const double* src, double* dst, DevState* st,
                              cudaStream_t s) {
  if (dd.ex != sd.ex || dd.ey != sd.ey || dd.ez != sd.ez || dd.g != sd.g || dd.px < sd.px)
    return cudaErrorInvalidValue;
  const long long rows = (long long)sd.ey * sd.ez;
  k_copy_guess<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(dd, sd, src, dst, st);
  return cudaGetLastError();
}

// Set-up pass of FP64 solves: fs = factor * rho on interior nodes and, in the
// same sweep, the partials of the reference norm ||f - A phi0||, phi0 = the
// boundary data of phi with every interior value read as zero.  The value at
// a node is fs plus c * phi over its boundary neighbours, added axis by axis
// (x, then y, then z; per axis the offsets o = 1..G in turn, each term one FMA
// of a selected ghost value): away from the boundary it is fs itself, and the
// pass costs one FP64 multiply and one FMA per node.  The x terms run in the
// warps that hold a lane next to an x boundary (all lanes of such a warp add
// the term, zero where it does not apply, so no lane walks alone); the y and
// z terms are uniform over a warp.  The max |value| runs on the integer pipe.
template <int G>
__device__ __forceinline__ double add_ghost_terms(double v, const double* __restrict__ phi, long long p,
                                                  long long stride, int a, int n, const Coef<double>& cf,
                                                  int axis) {
  // a = array index along the axis; interior [G, G + n - 1]
#pragma unroll
  for (int o = 1; o <= G; o++) {
    const bool lo = a - o < G, hi = a + o > G + n - 1;
    const double c = o == 1 ? cf.c1[axis] : cf.c2[axis];
    if (n >= 2 * o) {
      // one side at most (the node would need n < 2o to see both ghosts)
      const double b = lo ? phi[p - o * stride] : (hi ? phi[p + o * stride] : 0.0);
      v = fma(b, c, v);
    } else {
      const double b = (lo ? phi[p - o * stride] : 0.0) + (hi ? phi[p + o * stride] : 0.0);
      v = fma(b, c, v);
    }
  }
  return v;
}

template <int G>
__global__ void __launch_bounds__(BX* BY)
    k_scale_rhs_ref(Dims d, Dims du, double factor, Coef<double> cf, const double* __restrict__ rho,
                    const double* __restrict__ phi, double* __restrict__ fs, double* __restrict__ partials) {
  const int i = blockIdx.x * BX + threadIdx.x + G;
  const int j = blockIdx.y * BY + threadIdx.y + G;
  const int zc = zchunk(d.nk());
  const int k0 = blockIdx.z * zc + G;
  const int k1 = min(k0 + zc, G + d.nk());
  const int ni = d.ni(), nj = d.nj(), nk = d.nk();
  const bool act = i < G + ni && j < G + nj;
  // the warp holds a lane next to an x boundary (decided once, warp-uniform)
  const bool wx = __any_sync(0xffffffffu, act && (i < 2 * G || i >= ni));
  const bool yb = j < 2 * G || j >= nj;
  double s2 = 0.0;
  AbsMax mx;
  if (act) {
    const long long syu = du.sy(), szu = du.sz();
    for (int k = k0; k < k1; k++) {
      const long long pu = du.at(i, j, k);
      const double f = factor * rho[pu];
      fs[d.at(i, j, k)] = f;
      double v = f;
      if (wx) v = add_ghost_terms<G>(v, phi, pu, 1, i, ni, cf, 0);
      if (yb) v = add_ghost_terms<G>(v, phi, pu, syu, j, nj, cf, 1);
      if (k < 2 * G || k >= nk) v = add_ghost_terms<G>(v, phi, pu, szu, k, nk, cf, 2);
      s2 = fma(v, v, s2);
      mx.take(v);
    }
  }
  block_sum_max(s2, mx.value(), partials);
}

cudaError_t launch_scale_rhs_ref(const Dims& d, const Dims& du, int order, const double h[3], double factor,
                                 const double* rho, const double* phi, double* fs, double* partials,
                                 cudaStream_t s) {
  if (du.ex != d.ex || du.ey != d.ey || du.ez != d.ez || du.g != d.g || d.g != order / 2)
    return cudaErrorInvalidValue;
  const Coef<double> cf = make_coef<double>(d, h, order);
  if (order == 2) k_scale_rhs_ref<1><<<point_grid(d), dim3(BX, BY), 0, s>>>(d, du, factor, cf, rho, phi, fs, partials);
  else k_scale_rhs_ref<2><<<point_grid(d), dim3(BX, BY), 0, s>>>(d, du, factor, cf, rho, phi, fs, partials);
  return cudaGetLastError();
}

template <int G, bool ISO, typename TI>
static cudaError_t delta_t(const Dims& d, const double h[3], int order, const void* phi,
                           const void* fs, int dout, void* out, double out_scale,
                           const DevState* st, bool zi, double* partials, cudaStream_t s) {
  using C = typename St<TI>::C;
  Coef<C> cf = make_coef<C>(d, h, order);
  // the refinement path needs max |delta| for its scale; plain norms need the sum only
  if (partials == nullptr)
    k_delta<G, ISO, TI, 0><<<point_grid(d), dim3(BX, BY), 0, s>>>(
        d, cf, (const TI*)phi, (const TI*)fs, dout, out, out_scale, st, zi ? 1 : 0, partials);
  else if (st != nullptr || zi)
    k_delta<G, ISO, TI, 2><<<point_grid(d), dim3(BX, BY), 0, s>>>(
        d, cf, (const TI*)phi, (const TI*)fs, dout, out, out_scale, st, zi ? 1 : 0, partials);
  else
    k_delta<G, ISO, TI, 1><<<point_grid(d), dim3(BX, BY), 0, s>>>(
        d, cf, (const TI*)phi, (const TI*)fs, dout, out, out_scale, st, zi ? 1 : 0, partials);
  return cudaGetLastError();
}

template <typename TI>
static cudaError_t delta_dispatch(const Dims& d, int order, const double h[3], const void* phi,
                                  const void* fs, int dout, void* out, double out_scale,
                                  const DevState* st, bool zi, double* partials, cudaStream_t s) {
  bool iso = is_iso(h);
  if (order == 2) {
    return iso ? delta_t<1, true, TI>(d, h, order, phi, fs, dout, out, out_scale, st, zi, partials, s)
               : delta_t<1, false, TI>(d, h, order, phi, fs, dout, out, out_scale, st, zi, partials, s);
  }
  return iso ? delta_t<2, true, TI>(d, h, order, phi, fs, dout, out, out_scale, st, zi, partials, s)
             : delta_t<2, false, TI>(d, h, order, phi, fs, dout, out, out_scale, st, zi, partials, s);
}

cudaError_t launch_delta_st(const Dims& d, int order, const double h[3], int din, const void* phi,
                            const void* fs, int dout, void* out, const DevState* st,
                            double* partials, cudaStream_t s) {
  if (din == DT_F64) return delta_dispatch<double>(d, order, h, phi, fs, dout, out, 1.0, st, false, partials, s);
  if (din == DT_F32) return delta_dispatch<float>(d, order, h, phi, fs, dout, out, 1.0, st, false, partials, s);
  return delta_dispatch<__nv_bfloat16>(d, order, h, phi, fs, dout, out, 1.0, st, false, partials, s);
}

cudaError_t launch_delta(const Dims& d, int order, const double h[3], int din, const void* phi,
                         const void* fs, int dout, void* out, double out_scale, bool zero_interior,
                         double* partials, LaunchCfg* cfg, cudaStream_t s) {
  if (cfg) cfg->nblocks = cart_partials_count(d);
  if (din == DT_F64)
    return delta_dispatch<double>(d, order, h, phi, fs, dout, out, out_scale, nullptr, zero_interior, partials, s);
  if (din == DT_F32)
    return delta_dispatch<float>(d, order, h, phi, fs, dout, out, out_scale, nullptr, zero_interior, partials, s);
  return delta_dispatch<__nv_bfloat16>(d, order, h, phi, fs, dout, out, out_scale, nullptr, zero_interior, partials, s);
}

// ------------------------------------------------------------------ delta after a sweep
// After a complete omega = 1 colour sweep, delta = phi_GS - phi is exactly zero on
// the last colour: its nodes were just set to phi_GS from operands that have not
// changed since, and this kernel repeats that arithmetic.  So delta is evaluated
// on the other colours only (one thread per node of each colour in a row, as in
// the colour passes) and zeros are stored on the last colour.
template <int G, bool ISO, typename T, typename TO>
__global__ void __launch_bounds__(BX* BY)
    k_delta_skip(Dims d, Coef<typename St<T>::C> cf, const T* __restrict__ phi,
                 const T* __restrict__ fs, TO* __restrict__ out) {
  using C = typename St<T>::C;
  using S = St<T>;
  constexpr int NCOL = G == 1 ? 2 : 3;
  const int t = blockIdx.x * BX + threadIdx.x;
  const int jn = blockIdx.y * BY + threadIdx.y + 1;
  if (jn > d.nj()) return;
  const int zc = zchunk(d.nk());
  const int kn0 = blockIdx.z * zc + 1;
  const int kn1 = min(kn0 + zc, d.nk() + 1);
  const long long sy = d.sy(), sz = d.sz();
  for (int kn = kn0; kn < kn1; kn++) {
#pragma unroll
    for (int colour = 0; colour < NCOL; colour++) {
      const int r0 = ((colour - jn - kn - 1) % NCOL + NCOL) % NCOL;
      const int in = 1 + r0 + NCOL * t;
      if (in > d.ni()) continue;
      const long long p = d.at(in + G - 1, jn + G - 1, kn + G - 1);
      if (colour == NCOL - 1) {
        St<TO>::st(out + p, (typename St<TO>::C)0);
      } else {
        const C dl = gs_value<G, ISO>(phi, p, sy, sz, cf, S::ld(fs + p)) - S::ld(phi + p);
        St<TO>::st(out + p, (typename St<TO>::C)dl);
      }
    }
  }
}

// FP64 7-point on equal spacings: delta on the red nodes along (j, k)
// diagonals (5 + 1 FP64 instructions per node, the order of k_sweep_diag) and
// zero on the black member of each pair.
__global__ void __launch_bounds__(BX* BY)
    k_delta_skip_diag(Dims d, double c1, const double* __restrict__ phi, const double* __restrict__ fs,
                      int dl, double* __restrict__ out) {
  const int t = blockIdx.x * BX + threadIdx.x;
  const int jn0 = blockIdx.y * BY + threadIdx.y + 2 - dl;
  const int kn0 = blockIdx.z * dl + 1;
  const int ni = d.ni(), nj = d.nj(), nk = d.nk();
  const int u0 = jn0 < 1 ? 1 - jn0 : 0;
  const int u1 = min(dl, min(nj - jn0 + 1, nk - kn0 + 1));
  if (u0 >= u1) return;
  const int p = (1 + jn0 + kn0) & 1;            // red member of the pair
  const int in = 1 + 2 * t + p, ib = 1 + 2 * t + (1 - p);
  if (in > ni && ib > ni) return;
  const long long sy = d.sy(), sz = d.sz(), step = sy + sz;
  long long c = d.at(in, jn0 + u0, kn0 + u0);
  const long long cb = ib - in;                 // offset of the black member
  if (in > ni) {   // only the black member is interior
    if (ib <= ni)
      for (int u = u0; u < u1; u++, c += step) out[c + cb] = 0.0;
    return;
  }
  double qprev = phi[c - sy] + phi[c - sz];
  // raw operands one node ahead, summed one step later (as in k_sweep_diag)
  double e = phi[c + 1], w = phi[c - 1], nn = phi[c + sy], up = phi[c + sz], f = fs[c], x = phi[c];
  for (int u = u0; u < u1; u++) {
    const long long cn = u + 1 < u1 ? c + step : c;
    const double e2 = phi[cn + 1], w2 = phi[cn - 1], n2 = phi[cn + sy], u2 = phi[cn + sz], f2 = fs[cn], x2 = phi[cn];
    const double q = nn + up;
    out[c] = fma(((e + w) + qprev) + q, c1, f) - x;
    qprev = q;
    if (ib <= ni) out[c + cb] = 0.0;
    c += step;
    e = e2;
    w = w2;
    nn = n2;
    up = u2;
    f = f2;
    x = x2;
  }
}

// FP64 7-point on equal spacings: delta on every node along (j, k) diagonals,
// both members of the thread's x pair, each with its carried (N + U) pair sum
// (5 + 1 FP64 instructions per node; the order of gs_value, so every delta
// equals k_delta's bit for bit and only the reductions run in another order).
// STORE: the refinement pass of k_delta (the scaled FP32/BF16 inner right-hand
// side, the FP32 sum of squares and max of the scaled values); otherwise the
// FP64 sum of delta^2.  Partials {sum, max} per block.  initial: the solve's
// initial residual; when the set-up copy found the guess's interior zero, the
// plain pass returns at once (its residual is the reference vector, whose norm
// is known) and the STORE pass takes delta = fs on every node away from the
// boundary, and one FMA of the ghost value on a face (the general formula on
// the rows and planes next to a y or z boundary): with the interior of phi
// zero these are the general path's deltas bit for bit (up to the sign of a
// zero), without its FP64 work.
template <bool STORE>
__global__ void __launch_bounds__(BX* BY)
    k_delta_diag(Dims d, double c1, const double* __restrict__ phi, const double* __restrict__ fs, int dl, int dout,
                 void* __restrict__ out, const DevState* __restrict__ st, int initial, double* __restrict__ partials) {
  const bool zero_guess = initial && st->guess_nonzero == 0;
  if (!STORE && zero_guess) return;
  const int t = blockIdx.x * BX + threadIdx.x;
  const int jn0 = blockIdx.y * BY + threadIdx.y + 2 - dl;
  const int kn0 = blockIdx.z * dl + 1;
  const int ni = d.ni(), nj = d.nj(), nk = d.nk();
  const int u0 = jn0 < 1 ? 1 - jn0 : 0;
  const int u1 = min(dl, min(nj - jn0 + 1, nk - kn0 + 1));
  const int ia = 1 + 2 * t;   // the pair (ia, ia + 1)
  double s2 = 0.0;
  float s2f = 0.0f, mxf = 0.0f;
  const double oscale = STORE ? st->scale_next : 1.0;
  const int oexp = pow2_exponent(oscale);
  auto take = [&](long long p, double dd) {
    if (STORE) {
      const float v = oexp != INT_MIN ? f64_to_f32_pow2(dd, oexp) : (float)(dd * oscale);
      s2f = fmaf(v, v, s2f);
      mxf = fmaxf(mxf, fabsf(v));
      if (dout == DT_F32) ((float*)out)[p] = v;
      else ((__nv_bfloat16*)out)[p] = __float2bfloat16_rn(v);
    } else {
      s2 = fma(dd, dd, s2);
    }
  };
  if (STORE && zero_guess) {
    if (u0 < u1 && ia <= ni) {
      const bool hb = ia + 1 <= ni;
      const long long sy = d.sy(), sz = d.sz(), step = sy + sz;
      long long c = d.at(ia, jn0 + u0, kn0 + u0);
      auto full = [&](long long p) {
        return fma(((phi[p + 1] + phi[p - 1]) + (phi[p - sy] + phi[p - sz])) + (phi[p + sy] + phi[p + sz]), c1,
                   fs[p]) - phi[p];
      };
      for (int u = u0; u < u1; u++, c += step) {
        const int j = jn0 + u, k = kn0 + u;
        if (j == 1 || j == nj || k == 1 || k == nk) {   // uniform over the warp
          take(c, full(c));
          if (hb) take(c + 1, full(c + 1));
          continue;
        }
        // x faces: the one nonzero neighbour is the ghost
        double va = fs[c];
        if (ia == 1) va = fma(phi[c - 1], c1, va);
        else if (ia == ni) va = fma(phi[c + 1], c1, va);
        take(c, va);
        if (hb) {
          double vb = fs[c + 1];
          if (ia + 1 == ni) vb = fma(phi[c + 2], c1, vb);
          take(c + 1, vb);
        }
      }
    }
  } else if (u0 < u1 && ia <= ni) {
    const bool hb = ia + 1 <= ni;
    const long long sy = d.sy(), sz = d.sz(), step = sy + sz;
    long long c = d.at(ia, jn0 + u0, kn0 + u0);
    const long long o = hb ? 1 : 0;   // the second member (or the first again, unused)
    double qa = phi[c - sy] + phi[c - sz];
    double qb = phi[c + o - sy] + phi[c + o - sz];
    // raw operands of both members one node ahead, summed one step later
    double w = phi[c - 1], xa = phi[c], xb = phi[c + 1], e = phi[c + 2];
    double na = phi[c + sy], ua = phi[c + sz], nb = phi[c + o + sy], ub = phi[c + o + sz];
    double fa = fs[c], fb = fs[c + o];
    for (int u = u0; u < u1; u++) {
      const long long cn = u + 1 < u1 ? c + step : c;
      const double w2 = phi[cn - 1], xa2 = phi[cn], xb2 = phi[cn + 1], e2 = phi[cn + 2];
      const double na2 = phi[cn + sy], ua2 = phi[cn + sz], nb2 = phi[cn + o + sy], ub2 = phi[cn + o + sz];
      const double fa2 = fs[cn], fb2 = fs[cn + o];
      const double qa2 = na + ua;
      take(c, fma(((xb + w) + qa) + qa2, c1, fa) - xa);
      qa = qa2;
      if (hb) {
        const double qb2 = nb + ub;
        take(c + 1, fma(((e + xa) + qb) + qb2, c1, fb) - xb);
        qb = qb2;
      }
      c += step;
      w = w2;
      xa = xa2;
      xb = xb2;
      e = e2;
      na = na2;
      ua = ua2;
      nb = nb2;
      ub = ub2;
      fa = fa2;
      fb = fb2;
    }
  }
  if (STORE) block_sum_max_scaled(s2f, mxf, oscale, partials);
  else block_sum_max(s2, 0.0, partials);
}

cudaError_t launch_delta_diag(const Dims& d, const double h[3], const double* phi, const double* fs, int dout,
                              void* out, const DevState* st, bool initial, double* partials, int* nblocks,
                              cudaStream_t s) {
  if (!is_iso(h) || d.g != 1 || (out != nullptr && (st == nullptr || (dout != DT_F32 && dout != DT_BF16))) ||
      (initial && st == nullptr))
    return cudaErrorInvalidValue;
  const Coef<double> cf = make_coef<double>(d, h, 2);
  const int dl = diag_walk_len(d.nk());
  const int pairs = (d.ni() + 1) / 2;
  const dim3 grid((pairs + BX - 1) / BX, (d.nj() + dl - 1 + BY - 1) / BY, (d.nk() + dl - 1) / dl);
  if (nblocks) *nblocks = (int)(grid.x * grid.y * grid.z);
  if (out != nullptr)
    k_delta_diag<true><<<grid, dim3(BX, BY), 0, s>>>(d, cf.c1[0], phi, fs, dl, dout, out, st, initial ? 1 : 0,
                                                      partials);
  else
    k_delta_diag<false><<<grid, dim3(BX, BY), 0, s>>>(d, cf.c1[0], phi, fs, dl, DT_F64, nullptr, st,
                                                       initial ? 1 : 0, partials);
  return cudaGetLastError();
}

// FP64 13-point residual passes on equal spacings along the (j, k)
// anti-diagonal walks of k_sweep_diag13 (every delta equals gs_value's bit for
// bit; only reductions run in another order), on colours 0 and 1 after a
// sweep whose last colour 2 has delta = 0.  A thread owns an x triple and walks
// its two members of colours 0 and 1, each with its carried pair sums.  MODE 0:
// sum of delta^2 (the norm after a sweep); 1: delta stored, zero stored on
// colour 2 (the residual before a restriction).
template <int MODE>
__global__ void __launch_bounds__(BX* BY)
    k_delta_diag13(Dims d, double c1, double c2, const double* __restrict__ phi, const double* __restrict__ fs,
                   int dl, int dout, void* __restrict__ out, const DevState* __restrict__ st,
                   double* __restrict__ partials) {
  static_assert(MODE == 0 || MODE == 1, "every-node passes use k_delta_diag13_all");
  constexpr int NM = 2;   // members evaluated: colours 0 and 1
  const int t = blockIdx.x * BX + threadIdx.x;
  const int jn0 = blockIdx.y * BY + threadIdx.y + 2 - dl;
  const int kr0 = blockIdx.z * dl + 1;
  const int ni = d.ni(), nj = d.nj(), nk = d.nk();
  const int u0 = jn0 < 1 ? 1 - jn0 : 0;
  const int u1 = min(dl, min(nj - jn0 + 1, nk - kr0 + 1));
  double s2 = 0.0;
  if (u0 < u1 && 1 + 3 * t <= ni) {
    const int jk = jn0 + nk + 1 - kr0;
    const long long sy = d.sy(), sz = d.sz(), step = sy - sz;
    const long long c0 = d.at(1, jn0 + u0 + 1, nk + 1 - (kr0 + u0) + 1);   // x node 0 of the first walk node
    long long cm[3];
    bool ok[3];
#pragma unroll
    for (int m = 0; m < 3; m++) {
      const int x = 1 + 3 * t + (((m - jk - 1) % 3) + 3) % 3;   // the member of colour m
      ok[m] = x <= ni;
      cm[m] = c0 + (ok[m] ? x : 1 + 3 * t);
    }
    double su1[NM], su2[NM], su2n[NM], e1[NM], w1[NM], n1[NM], d1[NM], e2[NM], w2[NM], n2[NM], d2[NM], f[NM], xc[NM];
#pragma unroll
    for (int m = 0; m < NM; m++) {
      const long long c = cm[m];
      const long long c2n = u0 + 1 < u1 ? c + step : c;
      su1[m] = phi[c - sy] + phi[c + sz];
      su2[m] = phi[c - 2 * sy] + phi[c + 2 * sz];
      su2n[m] = phi[c2n - 2 * sy] + phi[c2n + 2 * sz];
      e1[m] = phi[c + 1]; w1[m] = phi[c - 1]; n1[m] = phi[c + sy]; d1[m] = phi[c - sz];
      e2[m] = phi[c + 2]; w2[m] = phi[c - 2]; n2[m] = phi[c + 2 * sy]; d2[m] = phi[c - 2 * sz];
      f[m] = fs[c]; xc[m] = phi[c];
    }
    for (int u = u0; u < u1; u++) {
      const bool more = u + 1 < u1;
#pragma unroll
      for (int m = 0; m < NM; m++) {
        const long long c = cm[m];
        const long long cn = more ? c + step : c;
        const double e1n = phi[cn + 1], w1n = phi[cn - 1], n1n = phi[cn + sy], d1n = phi[cn - sz];
        const double e2n = phi[cn + 2], w2n = phi[cn - 2], n2n = phi[cn + 2 * sy], d2n = phi[cn - 2 * sz];
        const double fn = fs[cn], xn = phi[cn];
        const double nd1 = n1[m] + d1[m], nd2 = n2[m] + d2[m];
        const double v1 = fma(((e1[m] + w1[m]) + su1[m]) + nd1, c1, f[m]);
        const double dl_ = fma(((e2[m] + w2[m]) + su2[m]) + nd2, c2, v1) - xc[m];
        if (ok[m]) {
          if (MODE == 1) ((double*)out)[c] = dl_;
          else s2 = fma(dl_, dl_, s2);
        }
        su1[m] = nd1;
        su2[m] = su2n[m];
        su2n[m] = nd2;
        cm[m] = cn;
        e1[m] = e1n; w1[m] = w1n; n1[m] = n1n; d1[m] = d1n;
        e2[m] = e2n; w2[m] = w2n; n2[m] = n2n; d2[m] = d2n;
        f[m] = fn; xc[m] = xn;
      }
      if (MODE == 1 && ok[2]) {   // the last colour: exactly zero after the sweep
        ((double*)out)[cm[2]] = 0.0;
        cm[2] += step;
      }
    }
  }
  if (MODE == 0) block_sum_max(s2, 0.0, partials);
}

// Every node (modes 2 and 3 of k_delta_diag13): one x per thread (consecutive
// lanes, consecutive x), one walk with its own carried pair sums; no lane is
// idle because every colour is evaluated.  !STORE with a state: the initial
// residual pass, skipped on a zero guess as in k_delta_diag.
template <bool STORE>
__global__ void __launch_bounds__(BX* BY)
    k_delta_diag13_all(Dims d, double c1, double c2, const double* __restrict__ phi, const double* __restrict__ fs,
                       int dl, int dout, void* __restrict__ out, const DevState* __restrict__ st,
                       double* __restrict__ partials) {
  if (!STORE && st != nullptr && st->guess_nonzero == 0) return;
  const int x = blockIdx.x * BX + threadIdx.x + 1;
  const int jn0 = blockIdx.y * BY + threadIdx.y + 2 - dl;
  const int kr0 = blockIdx.z * dl + 1;
  const int ni = d.ni(), nj = d.nj(), nk = d.nk();
  const int u0 = jn0 < 1 ? 1 - jn0 : 0;
  const int u1 = min(dl, min(nj - jn0 + 1, nk - kr0 + 1));
  double s2 = 0.0;
  float s2f = 0.0f, mxf = 0.0f;
  const double oscale = STORE ? st->scale_next : 1.0;
  const int oexp = pow2_exponent(oscale);
  if (u0 < u1 && x <= ni) {
    const long long sy = d.sy(), sz = d.sz(), step = sy - sz;
    long long c = d.at(x + 1, jn0 + u0 + 1, nk + 1 - (kr0 + u0) + 1);
    const long long c2n = u0 + 1 < u1 ? c + step : c;
    double su1 = phi[c - sy] + phi[c + sz];
    double su2 = phi[c - 2 * sy] + phi[c + 2 * sz];
    double su2n = phi[c2n - 2 * sy] + phi[c2n + 2 * sz];
    double e1 = phi[c + 1], w1 = phi[c - 1], n1 = phi[c + sy], d1 = phi[c - sz];
    double e2 = phi[c + 2], w2 = phi[c - 2], n2 = phi[c + 2 * sy], d2 = phi[c - 2 * sz];
    double f = fs[c], xc = phi[c];
    for (int u = u0; u < u1; u++) {
      const long long cn = u + 1 < u1 ? c + step : c;
      const double e1n = phi[cn + 1], w1n = phi[cn - 1], n1n = phi[cn + sy], d1n = phi[cn - sz];
      const double e2n = phi[cn + 2], w2n = phi[cn - 2], n2n = phi[cn + 2 * sy], d2n = phi[cn - 2 * sz];
      const double fn = fs[cn], xn = phi[cn];
      const double nd1 = n1 + d1, nd2 = n2 + d2;
      const double v1 = fma(((e1 + w1) + su1) + nd1, c1, f);
      const double dl_ = fma(((e2 + w2) + su2) + nd2, c2, v1) - xc;
      if (STORE) {
        const float v = oexp != INT_MIN ? f64_to_f32_pow2(dl_, oexp) : (float)(dl_ * oscale);
        s2f = fmaf(v, v, s2f);
        mxf = fmaxf(mxf, fabsf(v));
        if (dout == DT_F32) ((float*)out)[c] = v;
        else ((__nv_bfloat16*)out)[c] = __float2bfloat16_rn(v);
      } else {
        s2 = fma(dl_, dl_, s2);
      }
      su1 = nd1;
      su2 = su2n;
      su2n = nd2;
      c = cn;
      e1 = e1n; w1 = w1n; n1 = n1n; d1 = d1n;
      e2 = e2n; w2 = w2n; n2 = n2n; d2 = d2n;
      f = fn;
      xc = xn;
    }
  }
  if (STORE) block_sum_max_scaled(s2f, mxf, oscale, partials);
  else block_sum_max(s2, 0.0, partials);
}

static dim3 diag13_grid(const Dims& d, int* dl_out) {
  const int dl = diag_walk_len(d.nk());
  if (dl_out) *dl_out = dl;
  const int triples = (d.ni() + 2) / 3;
  return dim3((triples + BX - 1) / BX, (d.nj() + dl - 1 + BY - 1) / BY, (d.nk() + dl - 1) / dl);
}

static dim3 diag13_all_grid(const Dims& d) {
  const dim3 g = diag13_grid(d, nullptr);
  return dim3((d.ni() + BX - 1) / BX, g.y, g.z);
}

int delta_diag13_blocks(const Dims& d) {
  const dim3 g = diag13_all_grid(d);   // the larger of the two grids
  return (int)(g.x * g.y * g.z);
}

cudaError_t launch_delta_diag13(const Dims& d, const double h[3], int mode, const double* phi, const double* fs,
                                int dout, void* out, const DevState* st, double* partials, int* nblocks,
                                cudaStream_t s) {
  if (!is_iso(h) || d.g != 2 || mode < 0 || mode > 3 || (mode == 1 && out == nullptr) || (mode < 2 && st != nullptr) ||
      (mode == 3 && (out == nullptr || st == nullptr || (dout != DT_F32 && dout != DT_BF16))))
    return cudaErrorInvalidValue;
  const Coef<double> cf = make_coef<double>(d, h, 4);
  int dl = 0;
  const dim3 grid = diag13_grid(d, &dl), blk(BX, BY);
  if (nblocks) *nblocks = (int)(grid.x * grid.y * grid.z);
  const double a = cf.c1[0], b = cf.c2[0];
  switch (mode) {
    case 0: k_delta_diag13<0><<<grid, blk, 0, s>>>(d, a, b, phi, fs, dl, DT_F64, nullptr, nullptr, partials); break;
    case 1: k_delta_diag13<1><<<grid, blk, 0, s>>>(d, a, b, phi, fs, dl, DT_F64, out, nullptr, nullptr); break;
    case 2:
    case 3: {
      const dim3 ga = diag13_all_grid(d);
      if (nblocks) *nblocks = (int)(ga.x * ga.y * ga.z);
      if (mode == 2)
        k_delta_diag13_all<false><<<ga, blk, 0, s>>>(d, a, b, phi, fs, dl, DT_F64, nullptr, st, partials);
      else
        k_delta_diag13_all<true><<<ga, blk, 0, s>>>(d, a, b, phi, fs, dl, dout, out, st, partials);
      break;
    }
  }
  return cudaGetLastError();
}

template <int G, bool ISO, typename T, typename TO>
static cudaError_t delta_skip_t(const Dims& d, const double h[3], int order, const void* phi,
                                const void* fs, void* out, cudaStream_t s) {
  using C = typename St<T>::C;
  constexpr int NCOL = G == 1 ? 2 : 3;
  Coef<C> cf = make_coef<C>(d, h, order);
  if constexpr (G == 2 && ISO && sizeof(T) == 8 && sizeof(TO) == 8)
    return launch_delta_diag13(d, h, 1, (const double*)phi, (const double*)fs, DT_F64, out, nullptr, nullptr, nullptr, s);
  if constexpr (G == 1 && ISO && sizeof(T) == 8 && sizeof(TO) == 8) {
    const int dl = diag_walk_len(d.nk());
    const int pairs = (d.ni() + 1) / 2;
    const dim3 grid((pairs + BX - 1) / BX, (d.nj() + dl - 1 + BY - 1) / BY, (d.nk() + dl - 1) / dl);
    k_delta_skip_diag<<<grid, dim3(BX, BY), 0, s>>>(d, (double)cf.c1[0], (const double*)phi, (const double*)fs,
                                                     dl, (double*)out);
    return cudaGetLastError();
  }
  const int per_row = (d.ni() + NCOL - 1) / NCOL;
  const int gx = (per_row + BX - 1) / BX, gy = (d.nj() + BY - 1) / BY;
  const int zc = zchunk_for(gx * gy, d.nk());
  const dim3 grid(gx, gy, (d.nk() + zc - 1) / zc);
  k_delta_skip<G, ISO, T, TO><<<grid, dim3(BX, BY), 0, s>>>(d, cf, (const T*)phi, (const T*)fs, (TO*)out);
  return cudaGetLastError();
}

template <typename T, typename TO>
static cudaError_t delta_skip_dispatch(const Dims& d, int order, const double h[3], const void* phi,
                                       const void* fs, void* out, cudaStream_t s) {
  const bool iso = is_iso(h);
  if (order == 2)
    return iso ? delta_skip_t<1, true, T, TO>(d, h, order, phi, fs, out, s)
               : delta_skip_t<1, false, T, TO>(d, h, order, phi, fs, out, s);
  return iso ? delta_skip_t<2, true, T, TO>(d, h, order, phi, fs, out, s)
             : delta_skip_t<2, false, T, TO>(d, h, order, phi, fs, out, s);
}

cudaError_t launch_delta_after_sweep(const Dims& d, int order, const double h[3], int din, const void* phi,
                                     const void* fs, int dout, void* out, cudaStream_t s) {
  if (din == DT_F64 && dout == DT_F64) return delta_skip_dispatch<double, double>(d, order, h, phi, fs, out, s);
  if (din == DT_F32 && dout == DT_F32) return delta_skip_dispatch<float, float>(d, order, h, phi, fs, out, s);
  return cudaErrorNotSupported;
}

// ------------------------------------------------------------------ sweep (one colour)
// Nodes of colour c: (i+j+k) mod NCOL == c (global node indices).  Thread t of a
// row handles node i = i0 + NCOL t, i0 the first interior node of the colour.
template <int G, bool ISO, typename T, bool OM1>
__global__ void __launch_bounds__(BX* BY)
    k_sweep(Dims d, Coef<typename St<T>::C> cf, T* __restrict__ phi, const T* __restrict__ fs,
            int colour, typename St<T>::C omega, const DevState* __restrict__ st,
            const double* __restrict__ wtab, int wlen) {
  using C = typename St<T>::C;
  using S = St<T>;
  constexpr int NCOL = G == 1 ? 2 : 3;
  if (st != nullptr && st->done) return;
  // scheduled weights: colour pass n = NCOL * (completed steps) + colour of the
  // solve takes wtab[n] (the sequence of Eq. omega_n from n = 1), its last entry
  // once the sequence has reached its limit
  if (!OM1 && wtab != nullptr && st != nullptr) omega = (C)wtab[min(st->iter * NCOL + colour, wlen - 1)];
  const int t = blockIdx.x * BX + threadIdx.x;
  const int jn = blockIdx.y * BY + threadIdx.y + 1;
  if (jn > d.nj()) return;
  const int zc = zchunk(d.nk());
  const int kn0 = blockIdx.z * zc + 1;
  const int kn1 = min(kn0 + zc, d.nk() + 1);
  const long long sy = d.sy(), sz = d.sz();
  auto site = [&](int kn) -> long long {
    const int r0 = ((colour - jn - kn - 1) % NCOL + NCOL) % NCOL;
    const int in = 1 + r0 + NCOL * t;
    return in > d.ni() ? -1 : d.at(in + G - 1, jn + G - 1, kn + G - 1);
  };
  if constexpr (G == 1 && sizeof(T) == sizeof(double)) {
    // FP64 7-point: a colour point's neighbours all have the other colour and
    // are never written in this pass, so the operands of the next z point are
    // loaded before this point's store (two points' loads in flight).  (For
    // FP32/BF16 storage the plain loop measured faster.)
    struct Ops { C s6, f, c; };
    auto load = [&](long long p) -> Ops {
      Ops o;
      o.s6 = ((S::ld(phi + p + 1) + S::ld(phi + p - 1)) + (S::ld(phi + p + sy) + S::ld(phi + p - sy))) +
             (S::ld(phi + p + sz) + S::ld(phi + p - sz));
      o.f = S::ld(fs + p);
      o.c = OM1 ? (C)0 : S::ld(phi + p);
      return o;
    };
    long long p = kn0 < kn1 ? site(kn0) : -1;
    Ops cur{};
    if (p >= 0) cur = load(p);
    for (int kn = kn0; kn < kn1; kn++) {
      const long long pn = kn + 1 < kn1 ? site(kn + 1) : -1;
      Ops nxt{};
      if (pn >= 0) nxt = load(pn);
      if (p >= 0) {
        C gs;
        if (ISO) {
          gs = fma(cur.s6, cf.c1[0], cur.f);
        } else {
          gs = gs_value<G, ISO>(phi, p, sy, sz, cf, cur.f);
        }
        if (OM1) S::st(phi + p, gs);
        else S::st(phi + p, fma(omega, gs - cur.c, cur.c));
      }
      p = pn;
      cur = nxt;
    }
  } else {
    for (int kn = kn0; kn < kn1; kn++) {
      const long long p = site(kn);
      if (p < 0) continue;
      C gs = gs_value<G, ISO>(phi, p, sy, sz, cf, S::ld(fs + p));
      if (OM1) {
        S::st(phi + p, gs);
      } else {
        C old = S::ld(phi + p);
        S::st(phi + p, fma(omega, gs - old, old));
      }
    }
  }
}

// FP64 7-point colour pass on equal spacings along (j, k) diagonals.  Nodes
// (i, j + u, k + u) all have the same colour, and consecutive ones share two
// neighbours: the north + up pair b(j+1, k) + b(j, k+1) of one node is the
// south + down pair of the next.  A thread owns the x pair (1 + 2t, 2 + 2t),
// updates the member of the pass's colour (the same member along a diagonal)
// and walks DL nodes of one diagonal, carrying that pair sum:
// x_GS = c ((E + W) + (S + D) + (N + U)) + fs costs 5 FP64 instructions
// instead of 6.  a + b = b + a exactly, so the result does not depend on where
// a walk starts (the first node of a walk forms S + D itself).
template <bool OM1>
__global__ void __launch_bounds__(BX* BY)
    k_sweep_diag(Dims d, double c1, double* __restrict__ phi, const double* __restrict__ fs, int colour,
                 double omega, int dl, const DevState* __restrict__ st, const double* __restrict__ wtab,
                 int wlen) {
  if (st != nullptr && st->done) return;
  if (!OM1 && wtab != nullptr && st != nullptr) omega = wtab[min(st->iter * 2 + colour, wlen - 1)];
  const int t = blockIdx.x * BX + threadIdx.x;
  const int jn0 = blockIdx.y * BY + threadIdx.y + 2 - dl;   // walks start at jn0 = 2 - dl .. nj
  const int kn0 = blockIdx.z * dl + 1;
  const int ni = d.ni(), nj = d.nj(), nk = d.nk();
  // first interior node of the walk
  int u0 = jn0 < 1 ? 1 - jn0 : 0;
  const int u1 = min(dl, min(nj - jn0 + 1, nk - kn0 + 1));
  if (u0 >= u1) return;
  const int p = (colour + 1 + jn0 + kn0) & 1;   // the pair member of this colour on the whole diagonal
  const int in = 1 + 2 * t + p;
  if (in > ni) return;
  const long long sy = d.sy(), sz = d.sz(), step = sy + sz;
  long long c = d.at(in, jn0 + u0, kn0 + u0);
  double qprev = phi[c - sy] + phi[c - sz];
  // the next node's operands are loaded as raw values before this node's
  // arithmetic and store (its neighbours have the other colour and are not
  // written in this pass); their sums are formed one step later, so no
  // instruction of this step waits on them.  The last step reloads its own
  // node instead of branching.
  double e = phi[c + 1], w = phi[c - 1], nn = phi[c + sy], up = phi[c + sz], f = fs[c];
  double old = OM1 ? 0.0 : phi[c];
  for (int u = u0; u < u1; u++) {
    const long long cn = u + 1 < u1 ? c + step : c;
    const double e2 = phi[cn + 1], w2 = phi[cn - 1], n2 = phi[cn + sy], u2 = phi[cn + sz], f2 = fs[cn];
    const double old2 = OM1 ? 0.0 : phi[cn];
    const double q = nn + up;
    const double gs = fma(((e + w) + qprev) + q, c1, f);
    phi[c] = OM1 ? gs : fma(omega, gs - old, old);
    qprev = q;
    c += step;
    e = e2;
    w = w2;
    nn = n2;
    up = u2;
    f = f2;
    old = old2;
  }
}

// The first colour pass (colour 0, omega = 1) of a V-cycle on the finest FP64
// level (7-point, equal spacings), walked as k_sweep_diag walks it, with two
// additions for a convergence check that lags one pass behind the V-cycle it
// checks: the pass keeps the old value of every node it updates in save
// (packed at index c / 2: rows start at even offsets, so the colour-0 nodes of
// a row have distinct halves), so that the state before it can be put back,
// and with NORM it forms the block
// partials {sum of delta^2, 0}, delta = x_GS - x_old.  When the previous
// V-cycle ended with a complete sweep, colour 1's residual is exactly zero and
// these deltas (the operand order of the norm pass, so equal to its deltas bit
// for bit) are the whole residual of that V-cycle's result.  The variant
// without NORM opens a step: a plain pass that marks st->lag_pending = 1 for
// the restore (it saves nothing: a step runs at least one iteration, whose
// pass with NORM saves what the restore puts back).
template <bool NORM>
__global__ void __launch_bounds__(BX* BY)
    k_sweep_diag_lag(Dims d, double c1, double* __restrict__ phi, const double* __restrict__ fs,
                     double* __restrict__ save, int dl, DevState* __restrict__ st, double* __restrict__ partials) {
  if (st->done) return;   // uniform over the grid
  if (!NORM && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    st->lag_pending = 1;
  const int t = blockIdx.x * BX + threadIdx.x;
  const int jn0 = blockIdx.y * BY + threadIdx.y + 2 - dl;
  const int kn0 = blockIdx.z * dl + 1;
  const int ni = d.ni(), nj = d.nj(), nk = d.nk();
  const int u0 = jn0 < 1 ? 1 - jn0 : 0;
  const int u1 = min(dl, min(nj - jn0 + 1, nk - kn0 + 1));
  const int pm = (1 + jn0 + kn0) & 1;   // the pair member of colour 0 on this diagonal
  const int in = 1 + 2 * t + pm;
  double s2 = 0.0;
  if (u0 < u1 && in <= ni) {
    const long long sy = d.sy(), sz = d.sz(), step = sy + sz;
    long long c = d.at(in, jn0 + u0, kn0 + u0);
    double qprev = phi[c - sy] + phi[c - sz];
    double e = phi[c + 1], w = phi[c - 1], nn = phi[c + sy], up = phi[c + sz], f = fs[c], old = phi[c];
    for (int u = u0; u < u1; u++) {
      const long long cn = u + 1 < u1 ? c + step : c;
      const double e2 = phi[cn + 1], w2 = phi[cn - 1], n2 = phi[cn + sy], u2 = phi[cn + sz], f2 = fs[cn];
      const double old2 = phi[cn];
      const double q = nn + up;
      const double gs = fma(((e + w) + qprev) + q, c1, f);
      if (NORM) {
        const double dd = gs - old;
        s2 = fma(dd, dd, s2);
        save[c >> 1] = old;   // packed: consecutive lanes, consecutive doubles
      }
      phi[c] = gs;
      qprev = q;
      c += step;
      e = e2;
      w = w2;
      nn = n2;
      up = u2;
      f = f2;
      old = old2;
    }
  }
  if (NORM) block_sum_max(s2, 0.0, partials);
}

// Put back the colour-0 values that the last lagged first pass of this step
// saved (a no-op when none ran): the state of the last V-cycle checked.
__global__ void __launch_bounds__(BX* BY)
    k_restore_colour0(Dims d, double* __restrict__ phi, const double* __restrict__ save,
                      const DevState* __restrict__ st) {
  if (!st->lag_pending) return;
  const int i = blockIdx.x * BX + threadIdx.x + 1;
  const int j = blockIdx.y * BY + threadIdx.y + 1;
  if (i > d.ni() || j > d.nj()) return;
  const int zc = zchunk(d.nk());
  const int k0 = blockIdx.z * zc + 1, k1 = min(k0 + zc, d.nk() + 1);
  for (int k = k0 + ((i + j + k0) & 1); k < k1; k += 2) {
    const long long p = d.at(i, j, k);
    phi[p] = save[p >> 1];
  }
}

cudaError_t launch_sweep_lag(const Dims& d, const double h[3], double* phi, const double* fs, double* save,
                             bool norm, DevState* st, double* partials, int* nblocks, cudaStream_t s) {
  // the packed save index needs rows and planes at even offsets
  if (!is_iso(h) || d.g != 1 || (norm && partials == nullptr) || (d.sy() & 1) || (d.sz() & 1))
    return cudaErrorInvalidValue;
  const Coef<double> cf = make_coef<double>(d, h, 2);
  const int dl = diag_walk_len(d.nk());
  const int pairs = (d.ni() + 1) / 2;
  const dim3 grid((pairs + BX - 1) / BX, (d.nj() + dl - 1 + BY - 1) / BY, (d.nk() + dl - 1) / dl);
  if (nblocks) *nblocks = (int)(grid.x * grid.y * grid.z);
  if (norm) k_sweep_diag_lag<true><<<grid, dim3(BX, BY), 0, s>>>(d, cf.c1[0], phi, fs, save, dl, st, partials);
  else k_sweep_diag_lag<false><<<grid, dim3(BX, BY), 0, s>>>(d, cf.c1[0], phi, fs, save, dl, st, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_restore_colour0(const Dims& d, double* phi, const double* save, const DevState* st,
                                   cudaStream_t s) {
  if (d.g != 1 || (d.sy() & 1) || (d.sz() & 1)) return cudaErrorInvalidValue;
  k_restore_colour0<<<point_grid(d), dim3(BX, BY), 0, s>>>(d, phi, save, st);
  return cudaGetLastError();
}

// FP64 13-point colour pass on equal spacings along (j, k) anti-diagonals: the
// nodes (i, j+u, k-u) have one colour of the three, none of their neighbours
// is written in the pass, and the pair sum N + D (distance 1) of one node is
// the S + U of the next, the N + D at distance 2 the S + U of the node after
// that.  So x_GS = c1 ((E + W) + (S + U) + (N + D)) + c2 (... at distance 2)
// + fs costs 10 FP64 instructions instead of 12 (the order of gs_value).  A
// thread owns an x triple and updates the member of the pass's colour along a
// walk of dl nodes; walks tile (j, nk + 1 - k) as the 7-point walks tile
// (j, k).  Raw operands of the next node are loaded a step ahead.
template <bool OM1>
__global__ void __launch_bounds__(BX* BY)
    k_sweep_diag13(Dims d, double c1, double c2, double* __restrict__ phi, const double* __restrict__ fs,
                   int colour, double omega, int dl, const DevState* __restrict__ st,
                   const double* __restrict__ wtab, int wlen) {
  if (st != nullptr && st->done) return;
  if (!OM1 && wtab != nullptr && st != nullptr) omega = wtab[min(st->iter * 3 + colour, wlen - 1)];
  const int t = blockIdx.x * BX + threadIdx.x;
  const int jn0 = blockIdx.y * BY + threadIdx.y + 2 - dl;   // walks start at jn0 = 2 - dl .. nj
  const int kr0 = blockIdx.z * dl + 1;                       // k reflected: k = nk + 1 - kr
  const int ni = d.ni(), nj = d.nj(), nk = d.nk();
  const int u0 = jn0 < 1 ? 1 - jn0 : 0;
  const int u1 = min(dl, min(nj - jn0 + 1, nk - kr0 + 1));
  if (u0 >= u1) return;
  const int jk = jn0 + nk + 1 - kr0;   // j + k, fixed along the walk
  const int in = 1 + 3 * t + (((colour - jk - 1) % 3) + 3) % 3;
  if (in > ni) return;
  const long long sy = d.sy(), sz = d.sz(), step = sy - sz;
  long long c = d.at(in + 1, jn0 + u0 + 1, nk + 1 - (kr0 + u0) + 1);   // array index = node + 1
  // S + U of the first node (distance 1), and at distance 2 of the first two nodes
  double su1 = phi[c - sy] + phi[c + sz];
  const long long c2n = u0 + 1 < u1 ? c + step : c;
  double su2 = phi[c - 2 * sy] + phi[c + 2 * sz];
  double su2n = phi[c2n - 2 * sy] + phi[c2n + 2 * sz];
  double e1 = phi[c + 1], w1 = phi[c - 1], n1 = phi[c + sy], d1 = phi[c - sz];
  double e2 = phi[c + 2], w2 = phi[c - 2], n2 = phi[c + 2 * sy], d2 = phi[c - 2 * sz], f = fs[c];
  double old = OM1 ? 0.0 : phi[c];
  for (int u = u0; u < u1; u++) {
    const long long cn = u + 1 < u1 ? c + step : c;
    const double e1n = phi[cn + 1], w1n = phi[cn - 1], n1n = phi[cn + sy], d1n = phi[cn - sz];
    const double e2n = phi[cn + 2], w2n = phi[cn - 2], n2n = phi[cn + 2 * sy], d2n = phi[cn - 2 * sz];
    const double fn = fs[cn], oldn = OM1 ? 0.0 : phi[cn];
    const double nd1 = n1 + d1, nd2 = n2 + d2;
    const double v1 = fma(((e1 + w1) + su1) + nd1, c1, f);
    const double gs = fma(((e2 + w2) + su2) + nd2, c2, v1);
    phi[c] = OM1 ? gs : fma(omega, gs - old, old);
    su1 = nd1;
    su2 = su2n;
    su2n = nd2;
    c += step;
    e1 = e1n; w1 = w1n; n1 = n1n; d1 = d1n;
    e2 = e2n; w2 = w2n; n2 = n2n; d2 = d2n;
    f = fn;
    old = oldn;
  }
}

template <int G, bool ISO, typename T>
static cudaError_t sweep_t(const Dims& d, const double h[3], int order, void* phi, const void* fs,
                           int colour, double omega, const DevState* st, const double* wtab, int wlen,
                           cudaStream_t s) {
  using C = typename St<T>::C;
  constexpr int NCOL = G == 1 ? 2 : 3;
  Coef<C> cf = make_coef<C>(d, h, order);
  if constexpr (G == 1 && ISO && sizeof(T) == sizeof(double)) {
    // diagonal walks of dl nodes (any dl gives the same result)
    const int dl = diag_walk_len(d.nk());
    const int pairs = (d.ni() + 1) / 2;
    const dim3 grid((pairs + BX - 1) / BX, (d.nj() + dl - 1 + BY - 1) / BY, (d.nk() + dl - 1) / dl);
    if (omega == 1.0 && wtab == nullptr)
      k_sweep_diag<true><<<grid, dim3(BX, BY), 0, s>>>(d, (double)cf.c1[0], (double*)phi, (const double*)fs,
                                                        colour, omega, dl, st, nullptr, 0);
    else
      k_sweep_diag<false><<<grid, dim3(BX, BY), 0, s>>>(d, (double)cf.c1[0], (double*)phi, (const double*)fs,
                                                         colour, omega, dl, st, wtab, wlen);
    return cudaGetLastError();
  }
  if constexpr (G == 2 && ISO && sizeof(T) == sizeof(double)) {
    const int dl = diag_walk_len(d.nk());
    const int triples = (d.ni() + 2) / 3;
    const dim3 grid((triples + BX - 1) / BX, (d.nj() + dl - 1 + BY - 1) / BY, (d.nk() + dl - 1) / dl);
    if (omega == 1.0 && wtab == nullptr)
      k_sweep_diag13<true><<<grid, dim3(BX, BY), 0, s>>>(d, (double)cf.c1[0], (double)cf.c2[0], (double*)phi,
                                                          (const double*)fs, colour, omega, dl, st, nullptr, 0);
    else
      k_sweep_diag13<false><<<grid, dim3(BX, BY), 0, s>>>(d, (double)cf.c1[0], (double)cf.c2[0], (double*)phi,
                                                           (const double*)fs, colour, omega, dl, st, wtab, wlen);
    return cudaGetLastError();
  }
  int per_row = (d.ni() + NCOL - 1) / NCOL;
  const int gx = (per_row + BX - 1) / BX, gy = (d.nj() + BY - 1) / BY;
  const int zc = zchunk_for(gx * gy, d.nk());
  dim3 grid(gx, gy, (d.nk() + zc - 1) / zc);
  if (omega == 1.0 && wtab == nullptr)
    k_sweep<G, ISO, T, true><<<grid, dim3(BX, BY), 0, s>>>(d, cf, (T*)phi, (const T*)fs, colour, (C)omega, st, nullptr, 0);
  else
    k_sweep<G, ISO, T, false><<<grid, dim3(BX, BY), 0, s>>>(d, cf, (T*)phi, (const T*)fs, colour, (C)omega, st, wtab, wlen);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t sweep_dispatch(const Dims& d, int order, const double h[3], void* phi,
                                  const void* fs, int colour, double omega, const DevState* st,
                                  const double* wtab, int wlen, cudaStream_t s) {
  bool iso = is_iso(h);
  if (order == 2)
    return iso ? sweep_t<1, true, T>(d, h, order, phi, fs, colour, omega, st, wtab, wlen, s)
               : sweep_t<1, false, T>(d, h, order, phi, fs, colour, omega, st, wtab, wlen, s);
  return iso ? sweep_t<2, true, T>(d, h, order, phi, fs, colour, omega, st, wtab, wlen, s)
             : sweep_t<2, false, T>(d, h, order, phi, fs, colour, omega, st, wtab, wlen, s);
}

cudaError_t launch_sweep_colour(const Dims& d, int order, const double h[3], int dt, void* phi,
                                const void* fs, int colour, double omega, const DevState* st,
                                cudaStream_t s, const double* wtab, int wlen) {
  if (wtab != nullptr && (st == nullptr || wlen < 1)) return cudaErrorInvalidValue;
  if (dt == DT_F64) return sweep_dispatch<double>(d, order, h, phi, fs, colour, omega, st, wtab, wlen, s);
  if (dt == DT_F32) return sweep_dispatch<float>(d, order, h, phi, fs, colour, omega, st, wtab, wlen, s);
  return sweep_dispatch<__nv_bfloat16>(d, order, h, phi, fs, colour, omega, st, wtab, wlen, s);
}

// ------------------------------------------------------------------ restriction
// Full weighting (Sec. 2.1.3): coarse node I <- sum_{d in {-1,0,1}^3} w w w delta(2I+d),
// w = (1,2,1)/4, times `factor` (4 maps a fine scaled residual to the coarse
// scaled right-hand side because d_coarse = d_fine / 4).
template <typename TF, typename TC>
__global__ void __launch_bounds__(BX* BY)
    k_restrict(Dims fd, Dims cd, const TF* __restrict__ df, TC* __restrict__ fsc, double factor) {
  using CF = typename St<TF>::C;
  using CC = typename St<TC>::C;
  const int I = blockIdx.x * BX + threadIdx.x + 1;
  const int J = blockIdx.y * BY + threadIdx.y + 1;
  if (I > cd.ni() || J > cd.nj()) return;
  const int zc = zchunk(cd.nk());
  const int K0 = blockIdx.z * zc + 1;
  const int K1 = min(K0 + zc, cd.nk() + 1);
  const int g = fd.g;
  const long long sy = fd.sy(), sz = fd.sz();
  const CF sc = (CF)(factor / 64.0);
  // the (x, y)-weighted sum of fine plane 2K + 1 closes coarse plane K and opens
  // K + 1: computed once per thread and carried (same values, same order)
  auto plane_sum = [&](long long q0) -> CF {
    CF rows[3];
#pragma unroll
    for (int dy = -1; dy <= 1; dy++) {
      const long long q = q0 + dy * sy;
      rows[dy + 1] = (St<TF>::ld(df + q - 1) + St<TF>::ld(df + q + 1)) + (CF)2 * St<TF>::ld(df + q);
    }
    return (rows[0] + rows[2]) + (CF)2 * rows[1];
  };
  CF below = plane_sum(fd.at(2 * I + g - 1, 2 * J + g - 1, 2 * K0 + g - 2));
  for (int K = K0; K < K1; K++) {
    const long long c = fd.at(2 * I + g - 1, 2 * J + g - 1, 2 * K + g - 1);
    const CF mid = plane_sum(c), above = plane_sum(c + sz);
    CF acc = (below + above) + (CF)2 * mid;
    St<TC>::st(fsc + cd.at(I + g - 1, J + g - 1, K + g - 1), (CC)(acc * sc));
    below = above;
  }
}

template <typename TF, typename TC>
static cudaError_t restrict_t(const Dims& fine, const Dims& cd, const void* df, void* fsc, double factor,
                              cudaStream_t s) {
  dim3 grid = point_grid(cd);
  k_restrict<TF, TC><<<grid, dim3(BX, BY), 0, s>>>(fine, cd, (const TF*)df, (TC*)fsc, factor);
  return cudaGetLastError();
}

cudaError_t launch_restrict(const Dims& fine, const Dims& coarse, int dt_f, const void* delta_f, int dt_c, void* fs_c,
                            double factor, cudaStream_t s) {
  if (dt_c == DT_F64) {
    if (dt_f == DT_F64) return restrict_t<double, double>(fine, coarse, delta_f, fs_c, factor, s);
    if (dt_f == DT_F32) return restrict_t<float, double>(fine, coarse, delta_f, fs_c, factor, s);
    return restrict_t<__nv_bfloat16, double>(fine, coarse, delta_f, fs_c, factor, s);
  }
  if (dt_c == DT_F32) {
    if (dt_f == DT_F64) return restrict_t<double, float>(fine, coarse, delta_f, fs_c, factor, s);
    if (dt_f == DT_F32) return restrict_t<float, float>(fine, coarse, delta_f, fs_c, factor, s);
    return restrict_t<__nv_bfloat16, float>(fine, coarse, delta_f, fs_c, factor, s);
  }
  return cudaErrorInvalidValue;
}

// Full weighting of a residual that is zero on the black nodes.  A fine plane
// at odd offset from the coarse plane holds red values at (+-1, 0) and
// (0, +-1) around (2I, 2J), one at even offset at (0, 0) and (+-1, +-1).  With
// the zero terms dropped, k_restrict's plane sum of an odd-offset plane is
// (2 ym + 2 yp) + 2 (xm + xp) = 2 ((ym + yp) + (xm + xp)) exactly (scaling by
// 2 commutes with rounding), so the odd planes are carried as half sums and
// the factor 2 moves into the scale; the even plane's sum is
// (a + b) + 4 c.  The result equals k_restrict's up to the sign of zeros.
template <typename TF, typename TC>
__global__ void __launch_bounds__(BX* BY)
    k_restrict_red(Dims fd, Dims cd, const TF* __restrict__ df, TC* __restrict__ fsc, double factor) {
  using CF = typename St<TF>::C;
  using CC = typename St<TC>::C;
  const int I = blockIdx.x * BX + threadIdx.x + 1;
  const int J = blockIdx.y * BY + threadIdx.y + 1;
  if (I > cd.ni() || J > cd.nj()) return;
  const int zc = zchunk(cd.nk());
  const int K0 = blockIdx.z * zc + 1;
  const int K1 = min(K0 + zc, cd.nk() + 1);
  const int g = fd.g;
  const long long sy = fd.sy(), sz = fd.sz();
  const CF sc2 = (CF)(2.0 * (factor / 64.0));
  auto odd_half = [&](long long q) -> CF {
    return (St<TF>::ld(df + q - sy) + St<TF>::ld(df + q + sy)) + (St<TF>::ld(df + q - 1) + St<TF>::ld(df + q + 1));
  };
  CF below = odd_half(fd.at(2 * I + g - 1, 2 * J + g - 1, 2 * K0 + g - 2));
  for (int K = K0; K < K1; K++) {
    const long long c = fd.at(2 * I + g - 1, 2 * J + g - 1, 2 * K + g - 1);
    const CF a = St<TF>::ld(df + c - sy - 1) + St<TF>::ld(df + c - sy + 1);
    const CF b = St<TF>::ld(df + c + sy - 1) + St<TF>::ld(df + c + sy + 1);
    const CF even = fma((CF)4, St<TF>::ld(df + c), a + b);
    const CF above = odd_half(c + sz);
    St<TC>::st(fsc + cd.at(I + g - 1, J + g - 1, K + g - 1), (CC)(((below + above) + even) * sc2));
    below = above;
  }
}

cudaError_t launch_restrict_red(const Dims& fine, const Dims& coarse, int dt_f, const void* delta_f, int dt_c,
                                void* fs_c, double factor, cudaStream_t s) {
  const dim3 grid = point_grid(coarse), blk(BX, BY);
  if (dt_f == DT_F64 && dt_c == DT_F64)
    k_restrict_red<double, double><<<grid, blk, 0, s>>>(fine, coarse, (const double*)delta_f, (double*)fs_c, factor);
  else if (dt_f == DT_F32 && dt_c == DT_F32)
    k_restrict_red<float, float><<<grid, blk, 0, s>>>(fine, coarse, (const float*)delta_f, (float*)fs_c, factor);
  else if (dt_f == DT_F32 && dt_c == DT_F64)
    k_restrict_red<float, double><<<grid, blk, 0, s>>>(fine, coarse, (const float*)delta_f, (double*)fs_c, factor);
  else if (dt_f == DT_F64 && dt_c == DT_F32)
    k_restrict_red<double, float><<<grid, blk, 0, s>>>(fine, coarse, (const double*)delta_f, (float*)fs_c, factor);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ prolongation
// phi_fine += P e_coarse, P = 8 R^T (trilinear).  One thread per coarse cell
// (I..I+1, J..J+1, K..K+1): it loads the cell's 8 corner values once and
// updates the cell's fine nodes 2I+a, 2J+b, 2K+c (a,b,c in {0,1}) by separable
// interpolation (x, then y, then z; a node midway between two coarse nodes
// takes their mean).  Fine node 0 of an axis is the boundary and is skipped;
// coarse boundary values are zero.  Every interior fine node belongs to exactly
// one cell.
// Each thread marches its cell column along z; the 8 fine values of cell K + 1
// (and the coarse face above it) are loaded before cell K's results are
// stored, so a thread keeps two cells' loads in flight (the kernel is bound by
// memory latency, not by its arithmetic).
template <typename TC, typename TF>
__global__ void __launch_bounds__(BX* BY)
    k_prolong(Dims fd, Dims cd, const TC* __restrict__ ec, TF* __restrict__ phif) {
  using CF = typename St<TF>::C;
  const int I = blockIdx.x * BX + threadIdx.x;   // cell index 0 .. nc-1
  const int J = blockIdx.y * BY + threadIdx.y;
  if (I >= cd.nx || J >= cd.ny) return;
  const int zc = zchunk(cd.nz);
  const int K0 = blockIdx.z * zc, K1 = min(K0 + zc, cd.nz);
  const int g = fd.g;
  const long long csy = cd.sy(), csz = cd.sz();
  const long long fsy = fd.sy(), fsz = fd.sz();
  const CF half = (CF)0.5;
  // the corner values of a coarse plane's cell face: [y][x]
  auto load_face = [&](long long q0, CF (&c)[2][2]) {
#pragma unroll
    for (int y = 0; y < 2; y++) {
      c[y][0] = (CF)St<TC>::ld(ec + q0 + y * csy);
      c[y][1] = (CF)St<TC>::ld(ec + q0 + y * csy + 1);
    }
  };
  // the (x, y)-interpolated values of a face: [b][a]
  auto face = [&](const CF (&c)[2][2], CF (&v)[2][2]) {
    CF vx[2][2];   // [y][a]
#pragma unroll
    for (int y = 0; y < 2; y++) {
      vx[y][0] = c[y][0];
      vx[y][1] = half * (c[y][0] + c[y][1]);
    }
#pragma unroll
    for (int a = 0; a < 2; a++) {
      v[0][a] = vx[0][a];
      v[1][a] = half * (vx[0][a] + vx[1][a]);
    }
  };
  // fine values of cell K (index [cz][b][a]; nodes on the low boundary are not read)
  auto load_fine = [&](int K, CF (&f)[2][2][2]) {
    const long long f0 = fd.at(2 * I + g - 1, 2 * J + g - 1, 2 * K + g - 1);
#pragma unroll
    for (int cz = 0; cz < 2; cz++)
#pragma unroll
      for (int b = 0; b < 2; b++)
#pragma unroll
        for (int a = 0; a < 2; a++) {
          const bool skip = (cz == 0 && K == 0) || (b == 0 && J == 0) || (a == 0 && I == 0);
          f[cz][b][a] = skip ? (CF)0 : St<TF>::ld(phif + f0 + cz * fsz + b * fsy + a);
        }
  };
  // the top face of cell K is the bottom face of cell K + 1: computed once
  CF vy[2][2][2];   // [z][b][a]
  CF cn[2][2], fcur[2][2][2], fnext[2][2][2];
  {
    CF c0[2][2];
    load_face(cd.at(I + g - 1, J + g - 1, K0 + g - 1), c0);
    face(c0, vy[0]);
  }
  if (K0 < K1) {
    load_face(cd.at(I + g - 1, J + g - 1, K0 + g), cn);
    load_fine(K0, fcur);
  }
  for (int K = K0; K < K1; K++) {
    face(cn, vy[1]);
    if (K + 1 < K1) {   // next cell's operands, before this cell's stores
      load_face(cd.at(I + g - 1, J + g - 1, K + g + 1), cn);
      load_fine(K + 1, fnext);
    }
    const long long f0 = fd.at(2 * I + g - 1, 2 * J + g - 1, 2 * K + g - 1);
#pragma unroll
    for (int cz = 0; cz < 2; cz++) {
      if (cz == 0 && K == 0) continue;
#pragma unroll
      for (int b = 0; b < 2; b++) {
        if (b == 0 && J == 0) continue;
#pragma unroll
        for (int a = 0; a < 2; a++) {
          if (a == 0 && I == 0) continue;
          const CF v = cz == 0 ? vy[0][b][a] : half * (vy[0][b][a] + vy[1][b][a]);
          St<TF>::st(phif + f0 + cz * fsz + b * fsy + a, fcur[cz][b][a] + v);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < 2; b++)
#pragma unroll
      for (int a = 0; a < 2; a++) vy[0][b][a] = vy[1][b][a];
#pragma unroll
    for (int cz = 0; cz < 2; cz++)
#pragma unroll
      for (int b = 0; b < 2; b++)
#pragma unroll
        for (int a = 0; a < 2; a++) fcur[cz][b][a] = fnext[cz][b][a];
  }
}

template <typename TC, typename TF>
static cudaError_t prolong_t(const Dims& fine, const Dims& cd, const void* ec, void* phif, cudaStream_t s) {
  const int gx = (cd.nx + BX - 1) / BX, gy = (cd.ny + BY - 1) / BY;
  const int zc = zchunk_for(gx * gy, cd.nz);
  const dim3 grid(gx, gy, (cd.nz + zc - 1) / zc);
  k_prolong<TC, TF><<<grid, dim3(BX, BY), 0, s>>>(fine, cd, (const TC*)ec, (TF*)phif);
  return cudaGetLastError();
}

cudaError_t launch_prolong(const Dims& fine, const Dims& coarse, int dt_c, const void* e_c, int dt_f, void* phi_f,
                           cudaStream_t s) {
  if (dt_c == DT_F64) {
    if (dt_f == DT_F64) return prolong_t<double, double>(fine, coarse, e_c, phi_f, s);
    if (dt_f == DT_F32) return prolong_t<double, float>(fine, coarse, e_c, phi_f, s);
    return prolong_t<double, __nv_bfloat16>(fine, coarse, e_c, phi_f, s);
  }
  if (dt_c == DT_F32) {
    if (dt_f == DT_F64) return prolong_t<float, double>(fine, coarse, e_c, phi_f, s);
    if (dt_f == DT_F32) return prolong_t<float, float>(fine, coarse, e_c, phi_f, s);
    return prolong_t<float, __nv_bfloat16>(fine, coarse, e_c, phi_f, s);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ elementwise
template <typename T>
__global__ void __launch_bounds__(BX* BY)
    k_scale_rhs(Dims d, Dims du, double factor, const double* __restrict__ rho, T* __restrict__ fs) {
  const int g = d.g;
  const int i = blockIdx.x * BX + threadIdx.x + g;
  const int j = blockIdx.y * BY + threadIdx.y + g;
  if (i >= g + d.ni() || j >= g + d.nj()) return;
  const int zc = zchunk(d.nk());
  const int k0 = blockIdx.z * zc + g, k1 = min(k0 + zc, g + d.nk());
  for (int k = k0; k < k1; k++)
    St<T>::st(fs + d.at(i, j, k), (typename St<T>::C)(factor * rho[du.at(i, j, k)]));
}

cudaError_t launch_scale_rhs(const Dims& d, const Dims& du, double factor, const double* rho, int dt,
                             void* fs, cudaStream_t s) {
  if (dt == DT_F64) k_scale_rhs<double><<<point_grid(d), dim3(BX, BY), 0, s>>>(d, du, factor, rho, (double*)fs);
  else if (dt == DT_F32) k_scale_rhs<float><<<point_grid(d), dim3(BX, BY), 0, s>>>(d, du, factor, rho, (float*)fs);
  else k_scale_rhs<__nv_bfloat16><<<point_grid(d), dim3(BX, BY), 0, s>>>(d, du, factor, rho, (__nv_bfloat16*)fs);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(BX* BY)
    k_scale_any(Dims d, double factor, const T* __restrict__ f, T* __restrict__ fs) {
  const int g = d.g;
  const int i = blockIdx.x * BX + threadIdx.x + g;
  const int j = blockIdx.y * BY + threadIdx.y + g;
  if (i >= g + d.ni() || j >= g + d.nj()) return;
  const int zc = zchunk(d.nk());
  const int k0 = blockIdx.z * zc + g, k1 = min(k0 + zc, g + d.nk());
  for (int k = k0; k < k1; k++) {
    const long long p = d.at(i, j, k);
    St<T>::st(fs + p, (typename St<T>::C)(factor * (double)St<T>::ld(f + p)));
  }
}

cudaError_t launch_scale_rhs_any(const Dims& d, double factor, int dt, const void* f, void* fs,
                                 cudaStream_t s) {
  if (dt == DT_F64) k_scale_any<double><<<point_grid(d), dim3(BX, BY), 0, s>>>(d, factor, (const double*)f, (double*)fs);
  else if (dt == DT_F32) k_scale_any<float><<<point_grid(d), dim3(BX, BY), 0, s>>>(d, factor, (const float*)f, (float*)fs);
  else k_scale_any<__nv_bfloat16><<<point_grid(d), dim3(BX, BY), 0, s>>>(d, factor, (const __nv_bfloat16*)f, (__nv_bfloat16*)fs);
  return cudaGetLastError();
}

template <typename TE>
__global__ void __launch_bounds__(BX* BY)
    k_correct(Dims d, const TE* __restrict__ e, double inv_scale, double* __restrict__ phi,
              const DevState* __restrict__ st) {
  if (st != nullptr && st->done) return;
  double isc = inv_scale;
  if (st != nullptr) isc = inverse_scale(st->scale_cur);
  const int g = d.g;
  const int i = blockIdx.x * BX + threadIdx.x + g;
  const int j = blockIdx.y * BY + threadIdx.y + g;
  if (i >= g + d.ni() || j >= g + d.nj()) return;
  const int zc = zchunk(d.nk());
  const int k0 = blockIdx.z * zc + g, k1 = min(k0 + zc, g + d.nk());
  // FP32/BF16 corrections scaled by a power of two: the scaled value is built
  // on the integer pipe and one DADD remains (the same bits as the FMA)
  const int ie = sizeof(TE) < sizeof(double) ? pow2_exponent(isc) : INT_MIN;
  // unrolled: the loads of several planes in flight together
#pragma unroll 4
  for (int k = k0; k < k1; k++) {
    const long long p = d.at(i, j, k);
    if (ie != INT_MIN) phi[p] += f32_to_f64_pow2((float)St<TE>::ld(e + p), ie);
    else phi[p] = fma((double)St<TE>::ld(e + p), isc, phi[p]);
  }
}

cudaError_t launch_correct(const Dims& d, int dt_e, const void* e, double inv_scale, double* phi,
                           const DevState* st, cudaStream_t s) {
  if (dt_e == DT_F64) k_correct<double><<<point_grid(d), dim3(BX, BY), 0, s>>>(d, (const double*)e, inv_scale, phi, st);
  else if (dt_e == DT_F32) k_correct<float><<<point_grid(d), dim3(BX, BY), 0, s>>>(d, (const float*)e, inv_scale, phi, st);
  else k_correct<__nv_bfloat16><<<point_grid(d), dim3(BX, BY), 0, s>>>(d, (const __nv_bfloat16*)e, inv_scale, phi, st);
  return cudaGetLastError();
}

// out = A phi = d * (phi_GS(fs=0) - phi) * (-1) ... written directly:
// A phi = d * (sum c phi_nb - phi)
template <int G, bool ISO, typename T>
__global__ void __launch_bounds__(BX* BY)
    k_apply(Dims d, Coef<typename St<T>::C> cf, const T* __restrict__ phi, T* __restrict__ out) {
  using C = typename St<T>::C;
  const int i = blockIdx.x * BX + threadIdx.x + G;
  const int j = blockIdx.y * BY + threadIdx.y + G;
  if (i >= G + d.ni() || j >= G + d.nj()) return;
  const int zc = zchunk(d.nk());
  const int k0 = blockIdx.z * zc + G, k1 = min(k0 + zc, G + d.nk());
  const long long sy = d.sy(), sz = d.sz();
  const C dd = (C)cf.d;
  for (int k = k0; k < k1; k++) {
    const long long p = d.at(i, j, k);
    C v = gs_value<G, ISO>(phi, p, sy, sz, cf, (C)0) - St<T>::ld(phi + p);
    St<T>::st(out + p, v * dd);
  }
}

template <typename T>
static cudaError_t apply_dispatch(const Dims& d, int order, const double h[3], const void* phi,
                                  void* out, cudaStream_t s) {
  using C = typename St<T>::C;
  Coef<C> cf = make_coef<C>(d, h, order);
  bool iso = is_iso(h);
  dim3 grid = point_grid(d), blk(BX, BY);
  if (order == 2) {
    if (iso) k_apply<1, true, T><<<grid, blk, 0, s>>>(d, cf, (const T*)phi, (T*)out);
    else k_apply<1, false, T><<<grid, blk, 0, s>>>(d, cf, (const T*)phi, (T*)out);
  } else {
    if (iso) k_apply<2, true, T><<<grid, blk, 0, s>>>(d, cf, (const T*)phi, (T*)out);
    else k_apply<2, false, T><<<grid, blk, 0, s>>>(d, cf, (const T*)phi, (T*)out);
  }
  return cudaGetLastError();
}

cudaError_t launch_apply(const Dims& d, int order, const double h[3], int dt, const void* phi,
                         void* out, cudaStream_t s) {
  if (dt == DT_F64) return apply_dispatch<double>(d, order, h, phi, out, s);
  if (dt == DT_F32) return apply_dispatch<float>(d, order, h, phi, out, s);
  return apply_dispatch<__nv_bfloat16>(d, order, h, phi, out, s);
}

// ------------------------------------------------------------------ coarsest-level CG
template <int G, bool ISO, typename TF, typename TE, int PPT, int MAXT>
__global__ void __launch_bounds__(MAXT)
    k_coarse_cg(Dims d, Coef<double> cf, const TF* __restrict__ fs, TE* __restrict__ e,
                double tol, int max_iter, DevState* __restrict__ st) {
  extern __shared__ double p[];
  coarse_cg_block<G, ISO, TF, TE, PPT, MAXT>(d, cf, fs, e, tol, max_iter, st, p);
}

size_t coarse_cg_smem_bytes(const Dims& d) { return (size_t)d.size() * sizeof(double); }

template <int G, bool ISO, typename TF, typename TE>
static cudaError_t coarse_t(const Dims& d, const double h[3], int order, const void* fs, void* e,
                            double tol, int max_iter, DevState* st, cudaStream_t s) {
  Coef<double> cf = make_coef<double>(d, h, order);
  const size_t smem = coarse_cg_smem_bytes(d);
  const int nint = d.ni() * d.nj() * d.nk();
  int ppt = 1;
  while (ppt < 16 && (nint + ppt - 1) / ppt > 128) ppt *= 2;
  // up to 512 unknowns: 4 warps (one per SM sub-partition, each with its FP64
  // unit) with up to 4 unknowns per thread
  if (nint <= 512) ppt = (nint + 127) / 128;
  // very elongated coarsest levels (more than 16 x 256 unknowns): up to 1024 threads x 8
  const bool wide = (nint + ppt - 1) / ppt > 256;
  if (wide) ppt = 8;
  if ((nint + ppt - 1) / ppt > (wide ? 1024 : 256)) return cudaErrorInvalidValue;
  const int nthr = std::max(32, (((nint + ppt - 1) / ppt) + 31) / 32 * 32);
  cudaError_t err;
#define PS_COARSE_LAUNCH(P, MT)                                                               \
  {                                                                                           \
    auto kern = k_coarse_cg<G, ISO, TF, TE, P, MT>;                                           \
    if (smem > 48 * 1024 &&                                                                   \
        (err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                    (int)smem)) != cudaSuccess)                               \
      return err;                                                                             \
    kern<<<1, nthr, smem, s>>>(d, cf, (const TF*)fs, (TE*)e, tol, max_iter, st);              \
  }
  if (wide) PS_COARSE_LAUNCH(8, 1024)
  else if (ppt == 1) PS_COARSE_LAUNCH(1, 256)
  else if (ppt == 2) PS_COARSE_LAUNCH(2, 256)
  else if (ppt == 3) PS_COARSE_LAUNCH(3, 256)
  else if (ppt == 4) PS_COARSE_LAUNCH(4, 256)
  else if (ppt == 8) PS_COARSE_LAUNCH(8, 256)
  else PS_COARSE_LAUNCH(16, 256)
#undef PS_COARSE_LAUNCH
  return cudaGetLastError();
}

template <typename TF, typename TE>
static cudaError_t coarse_dispatch(const Dims& d, int order, const double h[3], const void* fs,
                                   void* e, double tol, int max_iter, DevState* st, cudaStream_t s) {
  bool iso = is_iso(h);
  if (order == 2)
    return iso ? coarse_t<1, true, TF, TE>(d, h, order, fs, e, tol, max_iter, st, s)
               : coarse_t<1, false, TF, TE>(d, h, order, fs, e, tol, max_iter, st, s);
  return iso ? coarse_t<2, true, TF, TE>(d, h, order, fs, e, tol, max_iter, st, s)
             : coarse_t<2, false, TF, TE>(d, h, order, fs, e, tol, max_iter, st, s);
}

cudaError_t launch_coarse_cg(const Dims& d, int order, const double h[3], int dt_fs,
                             const void* fs, int dt_e, void* e, double tol, int max_iter,
                             DevState* st, cudaStream_t s) {
  if (dt_fs == DT_F64 && dt_e == DT_F64) return coarse_dispatch<double, double>(d, order, h, fs, e, tol, max_iter, st, s);
  if (dt_fs == DT_F32 && dt_e == DT_F32) return coarse_dispatch<float, float>(d, order, h, fs, e, tol, max_iter, st, s);
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ norm finisher
__global__ void k_set_budget(DevState* st, int k) {
  st->chunk_end = st->iter + k;
  st->lag_pending = 0;
}

__global__ void k_init_state(DevState* st, double tol, int max_iter) {
  DevState z;
  memset(&z, 0, sizeof(z));
  z.tol = tol;
  z.max_iter = max_iter;
  z.scale_cur = 1.0;
  z.scale_next = 1.0;
  z.ref = 1.0;
  *st = z;
}

cudaError_t launch_init_state(DevState* st, double tol, int max_iter, cudaStream_t s) {
  k_init_state<<<1, 1, 0, s>>>(st, tol, max_iter);
  return cudaGetLastError();
}

// First node of a loop graph: open the while loop only if there is work left.
__global__ void k_loop_gate(const DevState* st, unsigned long long cond) {
  const unsigned int go = (st->done == DONE_NO && st->iter < st->chunk_end) ? 1u : 0u;
  cudaGraphSetConditional((cudaGraphConditionalHandle)cond, go);
}

cudaError_t launch_loop_gate(const DevState* st, unsigned long long cond, cudaStream_t s) {
  k_loop_gate<<<1, 1, 0, s>>>(st, cond);
  return cudaGetLastError();
}

// out[i] = x[i] * 2^e rounded to FP32 by the refinement residual's conversion
__global__ void k_pow2_to_f32(const double* __restrict__ x, long long n, int e, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = f64_to_f32_pow2(x[i], e);
}

// phi[i] += e[i] * 2^p: the refinement's correction step, the scaled value
// built on the integer pipe and one DADD
__global__ void k_add_pow2_f32(const float* __restrict__ e, long long n, int p, double* __restrict__ phi) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    phi[i] += f32_to_f64_pow2(e[i], p);
}

cudaError_t launch_add_pow2_f32(const float* e, long long n, int p, double* phi, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long want = (n + 255) / 256;
  const int blocks = (int)std::min<long long>(want, 8LL * device_sm_count());
  k_add_pow2_f32<<<blocks, 256, 0, s>>>(e, n, p, phi);
  return cudaGetLastError();
}

cudaError_t launch_pow2_to_f32(const double* x, long long n, int e, float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long want = (n + 255) / 256;
  const int blocks = (int)std::min<long long>(want, 8LL * device_sm_count());
  k_pow2_to_f32<<<blocks, 256, 0, s>>>(x, n, e, out);
  return cudaGetLastError();
}

cudaError_t launch_set_budget(DevState* st, int k, cudaStream_t s) {
  k_set_budget<<<1, 1, 0, s>>>(st, k);
  return cudaGetLastError();
}

__global__ void k_finish_norm(const double* __restrict__ partials, int nblocks, double dscale,
                              int mode, DevState* __restrict__ st, unsigned long long cond,
                              int chunk) {
  finish_norm_block(partials, nblocks, dscale, mode, st, cond, chunk);
}

cudaError_t launch_finish_norm(const double* partials, int nblocks, double dscale, int mode,
                               DevState* st, cudaStream_t s, unsigned long long cond, int chunk) {
  k_finish_norm<<<1, 1024, 0, s>>>(partials, nblocks, dscale, mode, st, cond, chunk);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ CG kernels (FP64)
// The SPD system is -A x = -(f - A b) (Sec. 2.1.2 needs A SPD): its residual
// is r_spd = -(f - A phi) = d * delta.
template <int G, bool ISO>
__global__ void __launch_bounds__(BX* BY)
    k_cg_init(Dims d, Coef<double> cf, const double* __restrict__ phi, const double* __restrict__ fs,
              double* __restrict__ r, double* __restrict__ p, double* __restrict__ partials) {
  const int i = blockIdx.x * BX + threadIdx.x + G;
  const int j = blockIdx.y * BY + threadIdx.y + G;
  const int zc = zchunk(d.nk());
  const int k0 = blockIdx.z * zc + G, k1 = min(k0 + zc, G + d.nk());
  const long long sy = d.sy(), sz = d.sz();
  double s2 = 0.0;
  if (i < G + d.ni() && j < G + d.nj()) {
    for (int k = k0; k < k1; k++) {
      const long long c = d.at(i, j, k);
      double v = cf.d * (gs_value<G, ISO>(phi, c, sy, sz, cf, fs[c]) - phi[c]);
      r[c] = v;
      p[c] = v;
      s2 = fma(v, v, s2);
    }
  }
  block_sum_max(s2, 0.0, partials);
}

template <int G, bool ISO>
__global__ void __launch_bounds__(BX* BY)
    k_cg_apply(Dims d, Coef<double> cf, const double* __restrict__ p, double* __restrict__ q,
               double* __restrict__ partials, const DevState* __restrict__ st) {
  if (st->done) return;
  const int i = blockIdx.x * BX + threadIdx.x + G;
  const int j = blockIdx.y * BY + threadIdx.y + G;
  const int zc = zchunk(d.nk());
  const int k0 = blockIdx.z * zc + G, k1 = min(k0 + zc, G + d.nk());
  const long long sy = d.sy(), sz = d.sz();
  double s2 = 0.0;
  if (i < G + d.ni() && j < G + d.nj()) {
    for (int k = k0; k < k1; k++) {
      const long long c = d.at(i, j, k);
      double pc = p[c];
      double v = cf.d * (pc - gs_value<G, ISO>(p, c, sy, sz, cf, 0.0));
      q[c] = v;
      s2 = fma(pc, v, s2);
    }
  }
  block_sum_max(s2, 0.0, partials);
}

__global__ void __launch_bounds__(BX* BY)
    k_cg_update(Dims d, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                const double* __restrict__ q, double* __restrict__ partials,
                const DevState* __restrict__ st) {
  if (st->done) return;
  const int g = d.g;
  const double alpha = st->alpha;
  const int i = blockIdx.x * BX + threadIdx.x + g;
  const int j = blockIdx.y * BY + threadIdx.y + g;
  const int zc = zchunk(d.nk());
  const int k0 = blockIdx.z * zc + g, k1 = min(k0 + zc, g + d.nk());
  double s2 = 0.0;
  if (i < g + d.ni() && j < g + d.nj()) {
    for (int k = k0; k < k1; k++) {
      const long long c = d.at(i, j, k);
      // x solves -A x = ..., i.e. the potential itself: phi += alpha p
      x[c] = fma(alpha, p[c], x[c]);
      double rv = fma(-alpha, q[c], r[c]);
      r[c] = rv;
      s2 = fma(rv, rv, s2);
    }
  }
  block_sum_max(s2, 0.0, partials);
}

__global__ void __launch_bounds__(BX* BY)
    k_cg_pupdate(Dims d, const double* __restrict__ r, double* __restrict__ p,
                 const DevState* __restrict__ st) {
  if (st->done) return;
  const int g = d.g;
  const double beta = st->beta;
  const int i = blockIdx.x * BX + threadIdx.x + g;
  const int j = blockIdx.y * BY + threadIdx.y + g;
  if (i >= g + d.ni() || j >= g + d.nj()) return;
  const int zc = zchunk(d.nk());
  const int k0 = blockIdx.z * zc + g, k1 = min(k0 + zc, g + d.nk());
  for (int k = k0; k < k1; k++) {
    const long long c = d.at(i, j, k);
    p[c] = fma(beta, p[c], r[c]);
  }
}

// ------------------------------------------------------------------ PCG preconditioner
// z = B^-1 r for the multicolour Gauss-Seidel preconditioner of Sec. 2.1.2 in
// its symmetric form B = (D + L) D^-1 (D + U) of -A_0 (colour order): colour
// passes on -A_0 z = r from z = 0, ascending, then descending without the
// repeated middle pass.  A pass sets z_p = r_p / d + sum c1 z_nb (the scaled
// Gauss-Seidel value) on the nodes of its colour.  Thread t of a row owns the
// NCOL consecutive nodes 1 + NCOL t .. NCOL t + NCOL, one of each colour.
// MODE 0: first pass (colour 0; the block's other nodes are set to 0);
// MODE 1: a later pass; MODE 2: the last pass (colour 0), which also sums r.z
// over the whole block (the other colours are final) into per-block partials.
template <int G, bool ISO, int MODE>
__global__ void __launch_bounds__(BX* BY)
    k_pcg_pass(Dims d, Coef<double> cf, const double* __restrict__ r, double* __restrict__ z,
               int colour, double* __restrict__ partials, const DevState* __restrict__ st) {
  constexpr int NCOL = G == 1 ? 2 : 3;
  if (st->done) return;   // uniform: the partials are not read either
  const int t = blockIdx.x * BX + threadIdx.x;
  const int jn = blockIdx.y * BY + threadIdx.y + 1;
  const int zc = zchunk(d.nk());
  const int kn0 = blockIdx.z * zc + 1;
  const int kn1 = min(kn0 + zc, d.nk() + 1);
  const long long sy = d.sy(), sz = d.sz();
  double s2 = 0.0;
  if (jn <= d.nj()) {
    for (int kn = kn0; kn < kn1; kn++) {
      const int r0 = ((colour - jn - kn - 1) % NCOL + NCOL) % NCOL;   // offset of the colour's node in the block
      const int in = 1 + r0 + NCOL * t;
      if (MODE == 0) {
#pragma unroll
        for (int m = 0; m < NCOL; m++) {
          const int ib = 1 + NCOL * t + m;
          if (ib > d.ni()) break;
          const long long p = d.at(ib + G - 1, jn + G - 1, kn + G - 1);
          z[p] = ib == in ? r[p] * cf.inv_d : 0.0;
        }
        continue;
      }
      if (in <= d.ni()) {
        const long long p = d.at(in + G - 1, jn + G - 1, kn + G - 1);
        z[p] = gs_value<G, ISO>(z, p, sy, sz, cf, r[p] * cf.inv_d);
      }
      if (MODE == 2) {
#pragma unroll
        for (int m = 0; m < NCOL; m++) {
          const int ib = 1 + NCOL * t + m;
          if (ib > d.ni()) break;
          const long long p = d.at(ib + G - 1, jn + G - 1, kn + G - 1);
          s2 = fma(r[p], z[p], s2);
        }
      }
    }
  }
  if (MODE == 2) block_sum_max(s2, 0.0, partials);
}

static dim3 pcg_grid(const Dims& d, int order) {
  const int ncol = order == 2 ? 2 : 3;
  const int per_row = (d.ni() + ncol - 1) / ncol;
  const int gx = (per_row + BX - 1) / BX, gy = (d.nj() + BY - 1) / BY;
  const int zc = zchunk_for(gx * gy, d.nk());
  return dim3(gx, gy, (d.nk() + zc - 1) / zc);
}

int pcg_partials_count(const Dims& d, int order) {
  const dim3 g = pcg_grid(d, order);
  return (int)(g.x * g.y * g.z);
}

template <int G, bool ISO>
static cudaError_t pcg_precond_t(const Dims& d, const Coef<double>& cf, const double* r, double* z,
                                 double* partials, const DevState* st, cudaStream_t s) {
  constexpr int NCOL = G == 1 ? 2 : 3;
  const dim3 grid = pcg_grid(d, 2 * G), blk(BX, BY);
  k_pcg_pass<G, ISO, 0><<<grid, blk, 0, s>>>(d, cf, r, z, 0, partials, st);
  for (int c = 1; c < NCOL; c++) k_pcg_pass<G, ISO, 1><<<grid, blk, 0, s>>>(d, cf, r, z, c, partials, st);
  for (int c = NCOL - 2; c >= 1; c--) k_pcg_pass<G, ISO, 1><<<grid, blk, 0, s>>>(d, cf, r, z, c, partials, st);
  k_pcg_pass<G, ISO, 2><<<grid, blk, 0, s>>>(d, cf, r, z, 0, partials, st);
  return cudaGetLastError();
}

cudaError_t launch_pcg_precond(const Dims& d, int order, const double h[3], const double* r, double* z,
                               double* partials, const DevState* st, cudaStream_t s) {
  const Coef<double> cf = make_coef<double>(d, h, order);
  const bool iso = is_iso(h);
  if (order == 2) return iso ? pcg_precond_t<1, true>(d, cf, r, z, partials, st, s)
                             : pcg_precond_t<1, false>(d, cf, r, z, partials, st, s);
  return iso ? pcg_precond_t<2, true>(d, cf, r, z, partials, st, s)
             : pcg_precond_t<2, false>(d, cf, r, z, partials, st, s);
}

int pcg_precond_kernels(int order) { return order == 2 ? 3 : 5; }

// which 0: alpha = rho / (p.q); 1: convergence check on r.r, then (CG) beta = rr/rho, rho = rr;
// 2: start (rho = rr, initial check); 3: convergence check only (PCG);
// 4: PCG beta = (r.z)/rho, rho = r.z; 5: PCG start, rho = r.z
__global__ void k_cg_scalar(const double* __restrict__ partials, int nblocks, int which,
                            DevState* __restrict__ st, unsigned long long cond, int chunk) {
  __shared__ double red[32];
  if (which != 2 && st->done) {
    if ((which == 1 || which == 3) && threadIdx.x == 0) set_loop(st, cond, chunk);
    return;
  }
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[2 * b];
  double a[1] = {s};
  block_sum<1>(a, red);
  if (threadIdx.x != 0) return;
  const double S = a[0];
  if (which == 0) {
    st->pq = S;
    st->alpha = st->rho / S;
  } else if (which == 1 || which == 3) {
    st->iter += 1;
    st->rr = S;
    double rel = sqrt(S) / st->ref;
    st->rel = rel;
    if (which == 1) {
      st->beta = S / st->rho;
      st->rho = S;
    }
    if (!isfinite(rel) || rel > 1e3 * fmax(st->rel0, 1.0)) st->done = DONE_DIVERGED;
    else if (rel <= st->tol) st->done = DONE_CONVERGED;
    else if (st->iter >= st->max_iter) st->done = DONE_MAXITER;
    set_loop(st, cond, chunk);
  } else if (which == 4) {
    st->beta = S / st->rho;
    st->rho = S;
  } else if (which == 5) {
    st->rho = S;
  } else {
    st->rho = S;
    st->rr = S;
    st->iter = 0;
    double rel = sqrt(S) / st->ref;
    st->rel = rel;
    st->rel0 = rel;
    st->done = rel <= st->tol ? DONE_CONVERGED : (st->max_iter <= 0 ? DONE_MAXITER : DONE_NO);
  }
}

cudaError_t launch_cg_init(const Dims& d, int order, const double h[3], const double* phi,
                           const double* fs, double* r, double* p, double* partials,
                           LaunchCfg* cfg, cudaStream_t s) {
  Coef<double> cf = make_coef<double>(d, h, order);
  if (cfg) cfg->nblocks = cart_partials_count(d);
  bool iso = is_iso(h);
  dim3 grid = point_grid(d), blk(BX, BY);
  if (order == 2) {
    if (iso) k_cg_init<1, true><<<grid, blk, 0, s>>>(d, cf, phi, fs, r, p, partials);
    else k_cg_init<1, false><<<grid, blk, 0, s>>>(d, cf, phi, fs, r, p, partials);
  } else {
    if (iso) k_cg_init<2, true><<<grid, blk, 0, s>>>(d, cf, phi, fs, r, p, partials);
    else k_cg_init<2, false><<<grid, blk, 0, s>>>(d, cf, phi, fs, r, p, partials);
  }
  return cudaGetLastError();
}

cudaError_t launch_cg_apply(const Dims& d, int order, const double h[3], const double* p,
                            double* q, double* partials, const DevState* st, cudaStream_t s) {
  Coef<double> cf = make_coef<double>(d, h, order);
  bool iso = is_iso(h);
  dim3 grid = point_grid(d), blk(BX, BY);
  if (order == 2) {
    if (iso) k_cg_apply<1, true><<<grid, blk, 0, s>>>(d, cf, p, q, partials, st);
    else k_cg_apply<1, false><<<grid, blk, 0, s>>>(d, cf, p, q, partials, st);
  } else {
    if (iso) k_cg_apply<2, true><<<grid, blk, 0, s>>>(d, cf, p, q, partials, st);
    else k_cg_apply<2, false><<<grid, blk, 0, s>>>(d, cf, p, q, partials, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_cg_update(const Dims& d, double* x, double* r, const double* p, const double* q,
                             double* partials, const DevState* st, cudaStream_t s) {
  k_cg_update<<<point_grid(d), dim3(BX, BY), 0, s>>>(d, x, r, p, q, partials, st);
  return cudaGetLastError();
}

cudaError_t launch_cg_pupdate(const Dims& d, const double* r, double* p, const DevState* st,
                              cudaStream_t s) {
  k_cg_pupdate<<<point_grid(d), dim3(BX, BY), 0, s>>>(d, r, p, st);
  return cudaGetLastError();
}

cudaError_t launch_cg_scalar(const double* partials, int nblocks, int which, DevState* st,
                             cudaStream_t s, unsigned long long cond, int chunk) {
  k_cg_scalar<<<1, 1024, 0, s>>>(partials, nblocks, which, st, cond, chunk);
  return cudaGetLastError();
}

}  // namespace ps
