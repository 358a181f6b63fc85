// Spherical grids: variable-coefficient Laplacian (Eq. 2), right-Jacobi
// BiCGSTAB (Sec. 2.1.2, van der Vorst's method as described by Saad, with the
// preconditioner B^-1 = diag(A)^-1 applied to vectors, never formed), and the
// multipole outer boundary (Sec. 2.2).
//
// Operator in flux form on nodes r_i, theta_j, phi_k:
//   L p = rad_p_i (p_{i+1} - p) - rad_m_i (p - p_{i-1})
//       + (1/r_i^2) [ th_p_j (p_{j+1} - p) - th_m_j (p - p_{j-1}) + ph_j (p_{k+1} - 2p + p_{k-1}) ]
//   rad_p_i = r_{i+1/2}^2 / ((r_{i+1}-r_i) r_i^2 (r_{i+1}-r_{i-1})/2)   (r_{-1} = 2 r_0 - r_1,
//   rad_m_i = r_{i-1/2}^2 / ((r_i-r_{i-1}) r_i^2 (r_{i+1}-r_{i-1})/2)    r_N = r_{N-1}^2/r_{N-2})
//   th_p_j = sin(t_{j+1/2}) / (sin t_j dt^2), th_m_j = sin(t_{j-1/2}) / (sin t_j dt^2),
//   ph_j = 1 / (sin^2 t_j dp^2); the face sines at the poles are zero.
// Inner Neumann: p_{-1} = p_1 (mirror); phi periodic; outer ghost = Dirichlet.
// The ghost slots of internal vectors are zero; mirror/periodic rules are
// applied by index, so no ghost fill pass is needed.
#include <cmath>
#include <vector>

#include "cart_kernels.cuh"
#include "spherical.cuh"

namespace ps {

static constexpr int SBX = 32, SBY = 8, MAXL = 16;

template <typename C> struct Tab {
  const C *rad_p, *rad_m, *inv_r2, *th_p, *th_m, *ph, *inv_diag;
};
template <typename C> static Tab<C> tab_of(const SphTables& t);
template <> Tab<double> tab_of<double>(const SphTables& t) {
  return {t.rad_p, t.rad_m, t.inv_r2, t.th_p, t.th_m, t.ph, t.inv_diag};
}
template <> Tab<float> tab_of<float>(const SphTables& t) {
  return {t.rad_pf, t.rad_mf, t.inv_r2f, t.th_pf, t.th_mf, t.phf, t.inv_diagf};
}

template <typename T, typename C>
__device__ __forceinline__ C sph_L(const SphDims& d, const Tab<C>& tb, const T* __restrict__ p,
                                   int i, int j, int k, long long c) {
  const long long sy = d.sy(), sz = d.sz();
  const C pc = (C)p[c];
  const C pim = (C)(i == 0 ? p[c + 1] : p[c - 1]);
  const C pip = (C)p[c + 1];
  const C pjm = j == 0 ? pc : (C)p[c - sy];
  const C pjp = j == d.nt - 1 ? pc : (C)p[c + sy];
  const C pkm = (C)(k == 0 ? p[c + (long long)(d.np - 1) * sz] : p[c - sz]);
  const C pkp = (C)(k == d.np - 1 ? p[c - (long long)(d.np - 1) * sz] : p[c + sz]);
  const C ang = fma(tb.th_p[j], pjp - pc, fma(-tb.th_m[j], pc - pjm, tb.ph[j] * ((pkp + pkm) - (C)2 * pc)));
  return fma(tb.rad_p[i], pip - pc, fma(-tb.rad_m[i], pc - pim, tb.inv_r2[i] * ang));
}

// partials: 2 sums per block
__device__ __forceinline__ void block_sum2(double a, double b, double* partials) {
  __shared__ double sh[64];
  double v[2] = {a, b};
  block_sum<2>(v, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int bid = block_linear_id();
    partials[2 * bid] = v[0];
    partials[2 * bid + 1] = v[1];
  }
}

static inline dim3 sph_grid(const SphDims& d) {
  return dim3((d.nr + SBX - 1) / SBX, (d.nt + SBY - 1) / SBY, d.np);
}

// ------------------------------------------------------------------ plain apply (FP64)
__global__ void __launch_bounds__(SBX* SBY)
    k_sph_apply(SphDims d, Tab<double> tb, const double* __restrict__ phi, double* __restrict__ out) {
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nr || j >= d.nt) return;
  const long long c = d.at(i, j, k);
  out[c] = sph_L<double, double>(d, tb, phi, i, j, k, c);
}

cudaError_t launch_sph_apply(const SphDims& d, const SphTables& t, const double* phi, double* out,
                             cudaStream_t s) {
  k_sph_apply<<<sph_grid(d), dim3(SBX, SBY), 0, s>>>(d, tab_of<double>(t), phi, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ BiCGSTAB kernels
template <typename T>
__global__ void __launch_bounds__(SBX* SBY)
    k_bicg_resid(SphDims d, Tab<typename St<T>::C> tb, int mode, const double* __restrict__ rho,
                 double fscale, const T* __restrict__ fin, const void* __restrict__ xv,
                 int x_is_f64, T* __restrict__ r, T* __restrict__ rhat, T* __restrict__ p,
                 T* __restrict__ phat, double* __restrict__ partials) {
  using C = typename St<T>::C;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  double s0 = 0.0, s1 = 0.0;
  if (i < d.nr && j < d.nt) {
    const long long c = d.at(i, j, k);
    const C f = rho != nullptr ? (C)(fscale * rho[c]) : (C)fin[c];
    C Lx;
    if (mode == 0) {
      // boundary part only: the outer ghost enters through rad_p at i = nr-1
      C g = 0;
      if (i == d.nr - 1)
        g = x_is_f64 ? (C)((const double*)xv)[c + 1] : (C)((const T*)xv)[c + 1];
      Lx = tb.rad_p[i] * g;
    } else {
      Lx = x_is_f64 ? sph_L<double, C>(d, tb, (const double*)xv, i, j, k, c)
                    : sph_L<T, C>(d, tb, (const T*)xv, i, j, k, c);
    }
    const C rv = f - Lx;
    s0 = (double)rv * (double)rv;
    s1 = s0;
    if (mode == 1) {
      r[c] = (T)rv;
      rhat[c] = (T)rv;
      p[c] = (T)rv;
      phat[c] = (T)(rv * tb.inv_diag[j * d.nr + i]);
    }
  }
  block_sum2(s0, s1, partials);
}

template <typename T>
__global__ void __launch_bounds__(SBX* SBY)
    k_bicg_apply(SphDims d, Tab<typename St<T>::C> tb, const T* __restrict__ src, T* __restrict__ dst,
                 const T* __restrict__ w1, int with_tt, double* __restrict__ partials,
                 const DevState* __restrict__ st, int skip_early) {
  using C = typename St<T>::C;
  if (st->done || (skip_early && st->early)) return;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  double s0 = 0.0, s1 = 0.0;
  if (i < d.nr && j < d.nt) {
    const long long c = d.at(i, j, k);
    const C v = sph_L<T, C>(d, tb, src, i, j, k, c);
    dst[c] = (T)v;
    const double vd = (double)v;
    s0 = vd * (double)w1[c];
    if (with_tt) s1 = vd * vd;
  }
  block_sum2(s0, s1, partials);
}

template <typename T>
__global__ void __launch_bounds__(SBX* SBY)
    k_bicg_s(SphDims d, Tab<typename St<T>::C> tb, const T* __restrict__ r, const T* __restrict__ v,
             T* __restrict__ sv, T* __restrict__ shat, double* __restrict__ partials,
             const DevState* __restrict__ st) {
  using C = typename St<T>::C;
  if (st->done) return;
  const C alpha = (C)st->alpha;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  double s0 = 0.0;
  if (i < d.nr && j < d.nt) {
    const long long c = d.at(i, j, k);
    const C s = fma(-alpha, (C)v[c], (C)r[c]);
    sv[c] = (T)s;
    shat[c] = (T)(s * tb.inv_diag[j * d.nr + i]);
    s0 = (double)s * (double)s;
  }
  block_sum2(s0, 0.0, partials);
}

template <typename T>
__global__ void __launch_bounds__(SBX* SBY)
    k_bicg_xr(SphDims d, void* __restrict__ xv, int x_is_f64, T* __restrict__ r,
              const T* __restrict__ rhat, const T* __restrict__ phat, const T* __restrict__ sv,
              const T* __restrict__ shat, const T* __restrict__ tv, double* __restrict__ partials,
              const DevState* __restrict__ st) {
  using C = typename St<T>::C;
  if (st->done) return;
  const int early = st->early;
  const double alpha = st->alpha, omega = st->omega;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  double s0 = 0.0, s1 = 0.0;
  if (i < d.nr && j < d.nt) {
    const long long c = d.at(i, j, k);
    double dx = alpha * (double)phat[c];
    if (!early) dx = fma(omega, (double)shat[c], dx);
    if (x_is_f64) ((double*)xv)[c] += dx;
    else ((T*)xv)[c] = (T)((C)((T*)xv)[c] + (C)dx);
    if (!early) {
      const C rv = fma(-(C)omega, (C)tv[c], (C)sv[c]);
      r[c] = (T)rv;
      s0 = (double)rv * (double)rv;
      s1 = (double)rv * (double)rhat[c];
    }
  }
  if (!early) block_sum2(s0, s1, partials);
}

template <typename T>
__global__ void __launch_bounds__(SBX* SBY)
    k_bicg_p(SphDims d, Tab<typename St<T>::C> tb, const T* __restrict__ r, T* __restrict__ p,
             const T* __restrict__ v, T* __restrict__ phat, const DevState* __restrict__ st) {
  using C = typename St<T>::C;
  if (st->done) return;
  const C beta = (C)st->beta, omega = (C)st->omega;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nr || j >= d.nt) return;
  const long long c = d.at(i, j, k);
  const C pv = fma(beta, fma(-omega, (C)v[c], (C)p[c]), (C)r[c]);
  p[c] = (T)pv;
  phat[c] = (T)(pv * tb.inv_diag[j * d.nr + i]);
}

// which: 0 alpha; 1 s-norm check; 2 omega; 3 r check + beta
__device__ __forceinline__ void bicg_set_loop(const DevState* st, unsigned long long cond, int chunk) {
  if (chunk > 0) {
    const unsigned int more = (st->done == DONE_NO && st->iter < st->chunk_end) ? 1u : 0u;
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond, more);
  }
}

__global__ void k_bicg_scalar(const double* __restrict__ partials, int nblk, int which,
                              DevState* __restrict__ st, unsigned long long cond, int chunk) {
  __shared__ double sh[64];
  if (st->done) {
    if (which == 3 && threadIdx.x == 0) bicg_set_loop(st, cond, chunk);
    return;
  }
  if ((which == 2) && st->early) return;
  if (which == 3 && st->early) {
    if (threadIdx.x == 0) {
      st->iter += 1;
      st->rel = sqrt(st->ss) / st->ref;
      st->done = DONE_CONVERGED;
      st->early = 0;
      bicg_set_loop(st, cond, chunk);
    }
    return;
  }
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
    a += partials[2 * q];
    b += partials[2 * q + 1];
  }
  double v[2] = {a, b};
  block_sum<2>(v, sh);
  if (threadIdx.x != 0) return;
  if (which == 0) {
    st->alpha = st->rho / v[0];
  } else if (which == 1) {
    st->ss = v[0];
    if (sqrt(v[0]) / st->ref <= st->tol) st->early = 1;
  } else if (which == 2) {
    st->ts = v[0];
    st->tt = v[1];
    st->omega = v[0] / v[1];
  } else {
    st->iter += 1;
    st->rr = v[0];
    const double rel = sqrt(v[0]) / st->ref;
    st->rel = rel;
    const double rho_new = v[1];
    st->beta = (rho_new / st->rho) * (st->alpha / st->omega);
    st->rho = rho_new;
    if (!isfinite(rel) || rel > 1e3 * fmax(st->rel0, 1.0)) st->done = DONE_DIVERGED;
    else if (rel <= st->tol) st->done = DONE_CONVERGED;
    else if (st->iter >= st->max_iter) st->done = DONE_MAXITER;
    bicg_set_loop(st, cond, chunk);
  }
}

__global__ void k_bicg_start(const double* __restrict__ partials, int nblk, int mode,
                             DevState* __restrict__ st) {
  __shared__ double sh[64];
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
    a += partials[2 * q];
    b += partials[2 * q + 1];
  }
  double v[2] = {a, b};
  block_sum<2>(v, sh);
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    const double ref = sqrt(v[0]);
    st->ref = ref > 0.0 ? ref : 1.0;
    st->amax = ref;
    return;
  }
  st->rr = v[0];
  st->rho = v[1];
  st->iter = 0;
  st->early = 0;
  const double rel = sqrt(v[0]) / st->ref;
  st->rel = rel;
  st->rel0 = rel;
  st->done = rel <= st->tol ? DONE_CONVERGED : (st->max_iter <= 0 ? DONE_MAXITER : DONE_NO);
  if (!isfinite(rel)) st->done = DONE_DIVERGED;
}

template <typename T>
static cudaError_t resid_t(const SphDims& d, const SphTables& t, int mode, const double* rho,
                           double fscale, const void* fin, const void* x, int x_is_f64, void* r,
                           void* rhat, void* p, void* phat, double* partials, cudaStream_t s) {
  using C = typename St<T>::C;
  k_bicg_resid<T><<<sph_grid(d), dim3(SBX, SBY), 0, s>>>(
      d, tab_of<C>(t), mode, rho, fscale, (const T*)fin, x, x_is_f64, (T*)r, (T*)rhat, (T*)p,
      (T*)phat, partials);
  return cudaGetLastError();
}

cudaError_t launch_bicg_resid(const SphDims& d, const SphTables& t, int dt, int mode,
                              const double* rho, double fscale, const void* fin, const void* x,
                              void* r, void* rhat, void* p, void* phat, double* partials, int* nblk,
                              cudaStream_t s) {
  dim3 g = sph_grid(d);
  if (nblk) *nblk = g.x * g.y * g.z;
  // x is the FP64 potential when the arithmetic is FP64 or when rho is given
  // (outer residual); the inner FP32 solve passes FP32 vectors.
  if (dt == DT_F64)
    return resid_t<double>(d, t, mode, rho, fscale, fin, x, 1, r, rhat, p, phat, partials, s);
  return resid_t<float>(d, t, mode, rho, fscale, fin, x, 0, r, rhat, p, phat, partials, s);
}

cudaError_t launch_bicg_start(const double* partials, int nblk, int mode, DevState* st,
                              cudaStream_t s) {
  k_bicg_start<<<1, 256, 0, s>>>(partials, nblk, mode, st);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t iter_t(const SphDims& d, const SphTables& t, void* x, int x_is_f64, void* r,
                          const void* rhat, void* p, void* phat, void* v, void* sv, void* shat,
                          void* tv, double* partials, DevState* st, cudaStream_t s,
                          unsigned long long cond, int chunk) {
  using C = typename St<T>::C;
  const Tab<C> tb = tab_of<C>(t);
  const dim3 g = sph_grid(d), b(SBX, SBY);
  const int nblk = g.x * g.y * g.z;
  k_bicg_apply<T><<<g, b, 0, s>>>(d, tb, (const T*)phat, (T*)v, (const T*)rhat, 0, partials, st, 0);
  k_bicg_scalar<<<1, 1024, 0, s>>>(partials, nblk, 0, st, 0ull, 0);
  k_bicg_s<T><<<g, b, 0, s>>>(d, tb, (const T*)r, (const T*)v, (T*)sv, (T*)shat, partials, st);
  k_bicg_scalar<<<1, 1024, 0, s>>>(partials, nblk, 1, st, 0ull, 0);
  k_bicg_apply<T><<<g, b, 0, s>>>(d, tb, (const T*)shat, (T*)tv, (const T*)sv, 1, partials, st, 1);
  k_bicg_scalar<<<1, 1024, 0, s>>>(partials, nblk, 2, st, 0ull, 0);
  k_bicg_xr<T><<<g, b, 0, s>>>(d, x, x_is_f64, (T*)r, (const T*)rhat, (const T*)phat, (const T*)sv,
                               (const T*)shat, (const T*)tv, partials, st);
  k_bicg_scalar<<<1, 1024, 0, s>>>(partials, nblk, 3, st, cond, chunk);
  k_bicg_p<T><<<g, b, 0, s>>>(d, tb, (const T*)r, (T*)p, (const T*)v, (T*)phat, st);
  return cudaGetLastError();
}

cudaError_t launch_bicg_iter(const SphDims& d, const SphTables& t, int dt, void* x, void* r,
                             const void* rhat, void* p, void* phat, void* v, void* sv, void* shat,
                             void* tv, double* partials, DevState* st, cudaStream_t s,
                             unsigned long long cond, int chunk) {
  if (dt == DT_F64) return iter_t<double>(d, t, x, 1, r, rhat, p, phat, v, sv, shat, tv, partials, st, s, cond, chunk);
  return iter_t<float>(d, t, x, 0, r, rhat, p, phat, v, sv, shat, tv, partials, st, s, cond, chunk);
}

// Iterative refinement: r = f - L x in FP64, stored as FP32 times st->scale_next.
__global__ void __launch_bounds__(SBX* SBY)
    k_sph_outer_resid(SphDims d, Tab<double> tb, const double* __restrict__ rho, double fscale,
                      const double* __restrict__ x, float* __restrict__ out,
                      const DevState* __restrict__ st, double* __restrict__ partials) {
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  const double sc = st->scale_next;
  double s0 = 0.0, s1 = 0.0;
  if (i < d.nr && j < d.nt) {
    const long long c = d.at(i, j, k);
    const double rv = fscale * rho[c] - sph_L<double, double>(d, tb, x, i, j, k, c);
    out[c] = (float)(rv * sc);
    s0 = rv * rv;
    s1 = fabs(rv);
  }
  // second slot: sum |r| is not needed; keep max |r| for the scale
  __shared__ double sh[64];
  double v[1] = {s0};
  block_sum<1>(v, sh);
  double m = warp_max(s1);
  __shared__ double mx[32];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  if ((tid & 31) == 0) mx[tid >> 5] = m;
  __syncthreads();
  if (tid == 0) {
    for (int w = 0; w < (int)(blockDim.x * blockDim.y + 31) / 32; w++) m = fmax(m, mx[w]);
    const int bid = block_linear_id();
    partials[2 * bid] = v[0];
    partials[2 * bid + 1] = m;
  }
}

cudaError_t launch_sph_outer_resid(const SphDims& d, const SphTables& t, const double* rho,
                                   double fscale, const double* x, float* out, const DevState* st,
                                   double* partials, int* nblk, cudaStream_t s) {
  dim3 g = sph_grid(d);
  if (nblk) *nblk = g.x * g.y * g.z;
  k_sph_outer_resid<<<g, dim3(SBX, SBY), 0, s>>>(d, tab_of<double>(t), rho, fscale, x, out, st, partials);
  return cudaGetLastError();
}

template <typename TE>
__global__ void __launch_bounds__(SBX* SBY)
    k_sph_correct(SphDims d, const TE* __restrict__ e, double inv_scale, double* __restrict__ x,
                  const DevState* __restrict__ st) {
  if (st != nullptr) inv_scale = 1.0 / st->scale_cur;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nr || j >= d.nt) return;
  const long long c = d.at(i, j, k);
  x[c] = fma((double)e[c], inv_scale, x[c]);
}

cudaError_t launch_sph_correct(const SphDims& d, int dt_e, const void* e, double* x,
                               const DevState* st, cudaStream_t s) {
  if (dt_e == DT_F64) k_sph_correct<double><<<sph_grid(d), dim3(SBX, SBY), 0, s>>>(d, (const double*)e, 1.0, x, st);
  else k_sph_correct<float><<<sph_grid(d), dim3(SBX, SBY), 0, s>>>(d, (const float*)e, 1.0, x, st);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ multipole
// Moments (Eq. outer_multipole) factor on the spherical grid: a phi-Fourier
// pass per (r, theta) line, then the theta-Legendre and r sums per (l, m).
template <int L>
__global__ void __launch_bounds__(128)
    k_sph_fourier(SphDims d, const double* __restrict__ rho, const double* __restrict__ cosT,
                  const double* __restrict__ sinT, double* __restrict__ Fc, double* __restrict__ Fs) {
  const int i = blockIdx.x * 128 + threadIdx.x, j = blockIdx.y;
  if (i >= d.nr) return;
  double ac[L + 1], as[L + 1];
#pragma unroll
  for (int m = 0; m <= L; m++) { ac[m] = 0.0; as[m] = 0.0; }
  for (int k = 0; k < d.np; k++) {
    const double v = rho[d.at(i, j, k)];
#pragma unroll
    for (int m = 0; m <= L; m++) {
      ac[m] = fma(v, cosT[m * d.np + k], ac[m]);
      as[m] = fma(v, sinT[m * d.np + k], as[m]);
    }
  }
#pragma unroll
  for (int m = 0; m <= L; m++) {
    Fc[((long long)m * d.nt + j) * d.nr + i] = ac[m];
    Fs[((long long)m * d.nt + j) * d.nr + i] = as[m];
  }
}

template <int L>
static void fourier_launch(const SphDims& d, const SphTables& t, const double* rho, cudaStream_t s) {
  k_sph_fourier<L><<<dim3((d.nr + 127) / 128, d.nt), 128, 0, s>>>(d, rho, t.cosT, t.sinT, t.Fc, t.Fs);
}

__global__ void __launch_bounds__(256)
    k_sph_moments(SphDims d, int L, const double* __restrict__ Pn, const double* __restrict__ sinth,
                  const double* __restrict__ Rw, const double* __restrict__ Fc,
                  const double* __restrict__ Fs, double* __restrict__ q) {
  __shared__ double sh[32];
  const int lm = blockIdx.x;
  int l = 0;
  while ((l + 1) * (l + 1) <= lm) l++;
  const int m = lm - l * l - l;
  const int am = m < 0 ? -m : m;
  const double* F = m < 0 ? Fs : Fc;
  const double* P = Pn + (long long)(l * (L + 1) + am) * d.nt;
  double acc = 0.0;
  for (int i = threadIdx.x; i < d.nr; i += blockDim.x) {
    double a = 0.0;
    for (int j = 0; j < d.nt; j++)
      a = fma(P[j] * sinth[j], F[((long long)am * d.nt + j) * d.nr + i], a);
    acc = fma(Rw[l * d.nr + i], a, acc);
  }
  double v[1] = {acc};
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) q[lm] = v[0];
}

__global__ void __launch_bounds__(256)
    k_sph_face(SphDims d, int L, double G, double rg, const double* __restrict__ q,
               const double* __restrict__ Pn, const double* __restrict__ cosT,
               const double* __restrict__ sinT, double* __restrict__ phi) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= d.nt * d.np) return;
  const int j = id % d.nt, k = id / d.nt;
  double acc = 0.0, rl = 1.0 / rg;
  const double ir = 1.0 / rg;
  for (int l = 0; l <= L; l++) {
    double s = 0.0;
    for (int m = -l; m <= l; m++) {
      const int am = m < 0 ? -m : m;
      const double ang = m < 0 ? sinT[am * d.np + k] : cosT[am * d.np + k];
      s = fma(q[l * l + l + m], Pn[(long long)(l * (L + 1) + am) * d.nt + j] * ang, s);
    }
    acc = fma(s, rl, acc);
    rl *= ir;
  }
  phi[d.at(d.nr, j, k)] = -G * acc;
}

cudaError_t launch_sph_moments(const SphDims& d, const SphTables& t, const double* rho,
                               cudaStream_t s) {
  const int L = t.lmax;
  if (L < 0 || L > MAXL) return cudaErrorInvalidValue;
  switch (L) {
    case 0: fourier_launch<0>(d, t, rho, s); break;
    case 1: fourier_launch<1>(d, t, rho, s); break;
    case 2: fourier_launch<2>(d, t, rho, s); break;
    case 3: fourier_launch<3>(d, t, rho, s); break;
    case 4: fourier_launch<4>(d, t, rho, s); break;
    case 5: fourier_launch<5>(d, t, rho, s); break;
    case 6: fourier_launch<6>(d, t, rho, s); break;
    case 7: fourier_launch<7>(d, t, rho, s); break;
    case 8: fourier_launch<8>(d, t, rho, s); break;
    case 9: fourier_launch<9>(d, t, rho, s); break;
    case 10: fourier_launch<10>(d, t, rho, s); break;
    case 11: fourier_launch<11>(d, t, rho, s); break;
    case 12: fourier_launch<12>(d, t, rho, s); break;
    case 13: fourier_launch<13>(d, t, rho, s); break;
    case 14: fourier_launch<14>(d, t, rho, s); break;
    case 15: fourier_launch<15>(d, t, rho, s); break;
    default: fourier_launch<16>(d, t, rho, s); break;
  }
  k_sph_moments<<<(L + 1) * (L + 1), 256, 0, s>>>(d, L, t.Pn, t.sinth, t.Rw, t.Fc, t.Fs, t.q);
  return cudaGetLastError();
}

cudaError_t launch_sph_face(const SphDims& d, const SphTables& t, double G, double* phi,
                            cudaStream_t s) {
  const int n = d.nt * d.np;
  k_sph_face<<<(n + 255) / 256, 256, 0, s>>>(d, t.lmax, G, t.r_ghost, t.q, t.Pn, t.cosT, t.sinT, phi);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ tables
template <typename T>
static cudaError_t upload(T** dst, const std::vector<T>& src, size_t* bytes) {
  cudaError_t e = cudaMalloc(dst, std::max<size_t>(1, src.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  *bytes += src.size() * sizeof(T);
  if (src.empty()) return cudaSuccess;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

static std::vector<float> to_f(const std::vector<double>& v) {
  return std::vector<float>(v.begin(), v.end());
}

cudaError_t sph_tables_build(const SphDims& d, const double* r, const double* th, const double* ph,
                             int lmax, SphTables* t) {
  const int nr = d.nr, nt = d.nt, np = d.np;
  std::vector<double> re(nr + 2);   // re[i+1] = r_i, i = -1..nr
  for (int i = 0; i < nr; i++) re[i + 1] = r[i];
  re[0] = 2.0 * r[0] - r[1];
  re[nr + 1] = r[nr - 1] * r[nr - 1] / r[nr - 2];
  std::vector<double> rp(nr), rm(nr), ir2(nr);
  for (int i = 0; i < nr; i++) {
    const double rim = re[i], ri = re[i + 1], rip = re[i + 2];
    const double half = 0.5 * (rip - rim);
    const double fp = 0.5 * (ri + rip), fm = 0.5 * (rim + ri);
    rp[i] = fp * fp / ((rip - ri) * ri * ri * half);
    rm[i] = fm * fm / ((ri - rim) * ri * ri * half);
    ir2[i] = 1.0 / (ri * ri);
  }
  const double dth = M_PI / nt, dph = 2.0 * M_PI / np;
  std::vector<double> sface(nt + 1);
  for (int j = 0; j <= nt; j++) sface[j] = std::sin(j * M_PI / nt);
  sface[0] = 0.0;
  sface[nt] = 0.0;
  std::vector<double> tp(nt), tm(nt), pp(nt), sth(nt);
  for (int j = 0; j < nt; j++) {
    const double sc = std::sin(th[j]);
    sth[j] = sc;
    tp[j] = sface[j + 1] / (sc * dth * dth);
    tm[j] = sface[j] / (sc * dth * dth);
    pp[j] = 1.0 / (sc * sc * dph * dph);
  }
  std::vector<double> idg((size_t)nr * nt);
  for (int j = 0; j < nt; j++)
    for (int i = 0; i < nr; i++) {
      const double dg = -rp[i] - rm[i] - ir2[i] * (tp[j] + tm[j] + 2.0 * pp[j]);
      idg[(size_t)j * nr + i] = 1.0 / dg;
    }
  t->bytes = 0;
  cudaError_t e;
  if ((e = upload(&t->rad_p, rp, &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->rad_m, rm, &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->inv_r2, ir2, &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->th_p, tp, &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->th_m, tm, &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->ph, pp, &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->inv_diag, idg, &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->rad_pf, to_f(rp), &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->rad_mf, to_f(rm), &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->inv_r2f, to_f(ir2), &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->th_pf, to_f(tp), &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->th_mf, to_f(tm), &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->phf, to_f(pp), &t->bytes)) != cudaSuccess) return e;
  if ((e = upload(&t->inv_diagf, to_f(idg), &t->bytes)) != cudaSuccess) return e;
  // multipole tables
  t->lmax = lmax;
  if (lmax >= 0) {
    const int W = lmax + 1;
    std::vector<double> ct((size_t)W * np), st((size_t)W * np);
    for (int m = 0; m < W; m++)
      for (int k = 0; k < np; k++) {
        ct[(size_t)m * np + k] = std::cos(m * ph[k]);
        st[(size_t)m * np + k] = std::sin(m * ph[k]);
      }
    MultipoleTables mt;
    build_multipole_tables(lmax, &mt);
    // normalised associated Legendre values nrm(l,m) P_l^m(cos t_j) (no Condon-Shortley phase)
    std::vector<double> Pn((size_t)W * W * nt, 0.0);
    for (int j = 0; j < nt; j++) {
      const double x = std::cos(th[j]), s = std::sin(th[j]);
      std::vector<double> P((size_t)W * W, 0.0);   // P[l*W+m]
      double pmm = 1.0;
      for (int m = 0; m < W; m++) {
        if (m > 0) pmm *= (2 * m - 1) * s;
        P[m * W + m] = pmm;
        if (m + 1 < W) P[(m + 1) * W + m] = (2 * m + 1) * x * pmm;
        for (int l = m + 2; l < W; l++)
          P[l * W + m] = mt.rec_a[l * W + m] * x * P[(l - 1) * W + m] -
                         mt.rec_b[l * W + m] * P[(l - 2) * W + m];
      }
      for (int l = 0; l < W; l++)
        for (int m = 0; m <= l; m++) Pn[((size_t)l * W + m) * nt + j] = mt.nrm[l * W + m] * P[l * W + m];
    }
    std::vector<double> Rw((size_t)W * nr);
    for (int i = 0; i < nr; i++) {
      const double dr = 0.5 * (re[i + 2] - re[i]);
      double rl = r[i] * r[i];
      for (int l = 0; l < W; l++) {
        Rw[(size_t)l * nr + i] = rl * dr * dth * dph;
        rl *= r[i];
      }
    }
    if ((e = upload(&t->cosT, ct, &t->bytes)) != cudaSuccess) return e;
    if ((e = upload(&t->sinT, st, &t->bytes)) != cudaSuccess) return e;
    if ((e = upload(&t->Pn, Pn, &t->bytes)) != cudaSuccess) return e;
    if ((e = upload(&t->Rw, Rw, &t->bytes)) != cudaSuccess) return e;
    if ((e = upload(&t->sinth, sth, &t->bytes)) != cudaSuccess) return e;
    size_t nf = (size_t)W * nt * nr;
    if ((e = cudaMalloc(&t->Fc, nf * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t->Fs, nf * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t->q, (size_t)W * W * sizeof(double))) != cudaSuccess) return e;
    t->bytes += (2 * nf + W * W) * sizeof(double);
  }
  t->r_ghost = re[nr + 1];
  return cudaSuccess;
}

void sph_tables_free(SphTables* t) {
  void* ptrs[] = {t->rad_p, t->rad_m, t->inv_r2, t->th_p, t->th_m, t->ph, t->inv_diag,
                  t->rad_pf, t->rad_mf, t->inv_r2f, t->th_pf, t->th_mf, t->phf, t->inv_diagf,
                  t->cosT, t->sinT, t->Pn, t->Rw, t->sinth, t->Fc, t->Fs, t->q};
  for (void* p : ptrs) cudaFree(p);
  *t = SphTables();
}

}  // namespace ps
