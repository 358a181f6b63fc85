// Spherical grids: variable-coefficient Laplacian (Eq. 2), right-Jacobi
// BiCGSTAB (Sec. 2.1.2, van der Vorst's method as described by Saad, with the
// preconditioner B^-1 = diag(A)^-1 applied to vectors, never formed; stopping
// on true residuals by Sleijpen and van der Vorst's residual replacement), and
// the multipole outer boundary (Sec. 2.2).
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

// FP32 (the refinement form's inner solves) works on the volume-scaled system
// V L e = V r: vol is V per (theta_j, r_i) and inv_diag is 1 / (V diag(L)).
template <typename C> struct Tab {
  const C *rad_p, *rad_m, *inv_r2, *th_p, *th_m, *ph, *inv_diag;
  const C* vol;   // FP32 only; nullptr for FP64
};
template <typename C> static Tab<C> tab_of(const SphTables& t);
template <> Tab<double> tab_of<double>(const SphTables& t) {
  return {t.rad_p, t.rad_m, t.inv_r2, t.th_p, t.th_m, t.ph, t.inv_diag, nullptr};
}
template <> Tab<float> tab_of<float>(const SphTables& t) {
  return {t.rad_pf, t.rad_mf, t.inv_r2f, t.th_pf, t.th_mf, t.phf, t.inv_diag_vf, t.volf};
}

template <typename T, typename C>
__device__ __forceinline__ C sph_L(const SphDims& d, const Tab<C>& tb, const T* __restrict__ p,
                                   int i, int j, int k, long long c) {
  const long long sy = d.sy(), sz = d.sz();
  const C pc = (C)p[c];
  const C pim = (C)(i == 0 && !d.inner_ghost ? p[c + 1] : p[c - 1]);
  const C pip = (C)p[c + 1];
  const C pjm = j == 0 ? pc : (C)p[c - sy];
  const C pjp = j == d.nt - 1 ? pc : (C)p[c + sy];
  const C pkm = (C)(k == 0 ? p[c + (long long)(d.np - 1) * sz] : p[c - sz]);
  const C pkp = (C)(k == d.np - 1 ? p[c - (long long)(d.np - 1) * sz] : p[c + sz]);
  // FP32 (the refinement's inner vectors): the phi term as a sum of differences,
  // so that its rounding is relative to the differences and not to |p| (the
  // coefficient ph_j / r_i^2 reaches 1e11 at the inner poles)
  C kk;
  if constexpr (sizeof(C) == 4) kk = (pkp - pc) + (pkm - pc);
  else kk = (pkp + pkm) - (C)2 * pc;
  const C ang = fma(tb.th_p[j], pjp - pc, fma(-tb.th_m[j], pc - pjm, tb.ph[j] * kk));
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

// partials {a, 0}: one sum per block (half the shuffle tree of block_sum2)
__device__ __forceinline__ void block_sum1(double a, double* partials) {
  __shared__ double sh[32];
  double v[1] = {a};
  block_sum<1>(v, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int bid = block_linear_id();
    partials[2 * bid] = v[0];
    partials[2 * bid + 1] = 0.0;
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

// ------------------------------------------------------------------ red-black SOR
// Thread (t, j, k) updates the node i = 2t + ((colour + j + k) & 1) of its row,
// the one of this colour.  The mirror ghost P_{-1} = P_1 and the periodic
// ghosts take values of nodes of the other colour (Nphi even), so a pass never
// reads a value it writes.
__global__ void __launch_bounds__(SBX* SBY)
    k_sph_sor(SphDims d, Tab<double> tb, double* __restrict__ x, const double* __restrict__ rho,
              double fscale, int colour, double omega, const double* __restrict__ wc,
              double* __restrict__ wn, const double* __restrict__ rj2, const DevState* __restrict__ st) {
  if (st != nullptr && st->done) return;
  const int t = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  if (j >= d.nt) return;
  const int i = 2 * t + ((colour + j + k) & 1);
  if (i >= d.nr) return;
  const long long c = d.at(i, j, k);
  const int q = j * d.nr + i;
  const double r = fscale * rho[c] - sph_L<double, double>(d, tb, x, i, j, k, c);
  const double w = wc != nullptr ? wc[q] : omega;
  x[c] = fma(w * r, tb.inv_diag[q], x[c]);
  // the first node of this colour in the column (i, j) advances its weight
  if (wn != nullptr && k == ((colour + i + j) & 1)) wn[q] = 1.0 / (1.0 - rj2[q] * w / 4.0);
}

__global__ void __launch_bounds__(SBX* SBY)
    k_sph_resnorm(SphDims d, Tab<double> tb, const double* __restrict__ x,
                  const double* __restrict__ rho, double fscale, double* __restrict__ partials) {
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  double r2 = 0.0;
  if (i < d.nr && j < d.nt) {
    const long long c = d.at(i, j, k);
    const double r = fscale * rho[c] - sph_L<double, double>(d, tb, x, i, j, k, c);
    r2 = r * r;
  }
  block_sum2(r2, 0.0, partials);
}

__global__ void k_sph_sor_weights(int n, const double* __restrict__ rj2, int chebyshev, double* __restrict__ w) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  w[q] = chebyshev ? 1.0 / (1.0 - rj2[q] / 2.0) : 2.0 / (1.0 + sqrt(1.0 - rj2[q]));
}

cudaError_t launch_sph_sor(const SphDims& d, const SphTables& t, double* x, const double* rho,
                           double fscale, int colour, double omega, const double* wc, double* wn,
                           const DevState* st, cudaStream_t s) {
  if (wn != nullptr && (wc == nullptr || t.rj2 == nullptr)) return cudaErrorInvalidValue;
  const int half = (d.nr + 1) / 2;
  const dim3 grid((half + SBX - 1) / SBX, (d.nt + SBY - 1) / SBY, d.np);
  k_sph_sor<<<grid, dim3(SBX, SBY), 0, s>>>(d, tab_of<double>(t), x, rho, fscale, colour, omega, wc, wn, t.rj2, st);
  return cudaGetLastError();
}

int sph_resnorm_blocks(const SphDims& d) {
  const dim3 g = sph_grid(d);
  return (int)(g.x * g.y * g.z);
}

cudaError_t launch_sph_resnorm(const SphDims& d, const SphTables& t, const double* x,
                               const double* rho, double fscale, double* partials, int* nblk,
                               cudaStream_t s) {
  k_sph_resnorm<<<sph_grid(d), dim3(SBX, SBY), 0, s>>>(d, tab_of<double>(t), x, rho, fscale, partials);
  if (nblk) *nblk = sph_resnorm_blocks(d);
  return cudaGetLastError();
}

cudaError_t launch_sph_sor_weights(const SphDims& d, const SphTables& t, int chebyshev, double* w,
                                   cudaStream_t s) {
  const int n = d.nr * d.nt;
  k_sph_sor_weights<<<(n + 255) / 256, 256, 0, s>>>(n, t.rj2, chebyshev, w);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ red-black SOR, scaled form
// A thread owns the node pair (2t, 2t+1) of row (j, k) for the k of its chunk
// of phi planes; in colour pass c it updates the member p = (c + j + k) & 1 of
// each pair (exactly one per row and plane).  The per-(j, i) coefficients of
// both members stay in registers for the whole chunk.  Per update: x_GS from
// five fused multiply-adds and one add, then x += w (x_GS - x): 8 FP64
// instructions (the flux form with a separate residual took about 16).
static constexpr int SOR_TX = 32, SOR_TY = 8, SOR_KC = 8;

__global__ void __launch_bounds__(256)
    k_sph_gs(SphDims d, const double* __restrict__ ac, const double* __restrict__ rho, double fscale,
             double* __restrict__ g) {
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nr || j >= d.nt) return;
  const long long c = d.at(i, j, k);
  g[c] = -(fscale * rho[c]) / ac[j * d.nr + i];
}

struct SorCoef {
  double bip, bim, bjp, bjm, bk, ac, w, rj2;
};

// MODE 0 (red pass): update x_GS = sum b x_nb + g in sum form (8 FP64
// instructions): its rounding, about ulp(x), is that of storing x.
// MODE 1 (black pass): update with delta = x_GS - x in difference form,
// sum b (x_nb - x) + g (12 instructions), whose rounding is relative to the
// differences, and accumulate the black residual after the update,
// r = a_c (x_new - x_GS) = a_c (w - 1) delta.
// MODE 2 (red residuals after the black pass): r = -a_c delta in difference form.
// The residual norm needs the difference form: in sum form its rounding,
// a_c ulp(x), reaches 1e-8 of ||b|| on graded grids whose pole coefficients
// reach 1e11, and SOR would stagnate there.
template <int MODE>
__global__ void __launch_bounds__(SOR_TX* SOR_TY)
    k_sph_sor2(SphDims d, const double* __restrict__ tab, double* __restrict__ x, const double* __restrict__ g,
               int colour, double omega, const double* __restrict__ wc, double* __restrict__ wn,
               const double* __restrict__ rj2, double* __restrict__ partials, const DevState* __restrict__ st) {
  if (st != nullptr && st->done) return;
  const int t = blockIdx.x * SOR_TX + threadIdx.x, j = blockIdx.y * SOR_TY + threadIdx.y;
  const int k0 = blockIdx.z * SOR_KC, k1 = min(k0 + SOR_KC, d.np);
  const long long nq = (long long)d.nr * d.nt;
  const long long sy = d.sy(), sz = d.sz(), wrap = (long long)(d.np - 1) * sz;
  double acc = 0.0;
  if (j < d.nt) {
    // both members' coefficients in registers (selected, never indexed, so
    // that they stay out of local memory)
    auto load = [&](int p) {
      SorCoef f;
      const int i = min(2 * t + p, d.nr - 1);
      const long long q = (long long)j * d.nr + i;
      f.bip = tab[q];
      f.bim = tab[nq + q];
      f.bjp = tab[2 * nq + q];
      f.bjm = tab[3 * nq + q];
      f.bk = tab[4 * nq + q];
      f.ac = tab[5 * nq + q];
      f.w = wc != nullptr ? wc[q] : omega;
      f.rj2 = wn != nullptr ? rj2[q] : 0.0;
      return f;
    };
    const SorCoef c0 = load(0), c1 = load(1);
    for (int k = k0; k < k1; k++) {
      const int p = (colour + j + k) & 1;
      const int i = 2 * t + p;
      if (i >= d.nr) continue;
      SorCoef f;
      f.bip = p ? c1.bip : c0.bip;
      f.bim = p ? c1.bim : c0.bim;
      f.bjp = p ? c1.bjp : c0.bjp;
      f.bjm = p ? c1.bjm : c0.bjm;
      f.bk = p ? c1.bk : c0.bk;
      f.ac = p ? c1.ac : c0.ac;
      f.w = p ? c1.w : c0.w;
      f.rj2 = p ? c1.rj2 : c0.rj2;
      const long long c = d.at(i, j, k);
      const double xc = x[c];
      const double xim = (i == 0 && !d.inner_ghost) ? x[c + 1] : x[c - 1];
      const double xip = x[c + 1];
      const double xjm = j == 0 ? xc : x[c - sy];
      const double xjp = j == d.nt - 1 ? xc : x[c + sy];
      const double xkm = k == 0 ? x[c + wrap] : x[c - sz];
      const double xkp = k == d.np - 1 ? x[c - wrap] : x[c + sz];
      double delta;
      if (MODE == 0) {
        double gsv = fma(f.bk, xkp + xkm, g[c]);
        gsv = fma(f.bjp, xjp, gsv);
        gsv = fma(f.bjm, xjm, gsv);
        gsv = fma(f.bip, xip, gsv);
        gsv = fma(f.bim, xim, gsv);
        delta = gsv - xc;
      } else {
        delta = fma(f.bk, (xkp - xc) + (xkm - xc), g[c]);
        delta = fma(f.bjp, xjp - xc, delta);
        delta = fma(f.bjm, xjm - xc, delta);
        delta = fma(f.bip, xip - xc, delta);
        delta = fma(f.bim, xim - xc, delta);
      }
      if (MODE == 2) {
        const double e = f.ac * delta;
        acc = fma(e, e, acc);
        continue;
      }
      x[c] = fma(f.w, delta, xc);
      if (MODE == 1) {
        const double e = (f.w - 1.0) * f.ac * delta;
        acc = fma(e, e, acc);
      }
      // the first node of this colour in the column (i, j) advances its weight
      if (wn != nullptr && k == ((colour + i + j) & 1)) wn[(long long)j * d.nr + i] = 1.0 / (1.0 - f.rj2 * f.w / 4.0);
    }
  }
  if (MODE != 0) block_sum2(acc, 0.0, partials);
}

static inline dim3 sor2_grid(const SphDims& d) {
  const int half = (d.nr + 1) / 2;
  return dim3((half + SOR_TX - 1) / SOR_TX, (d.nt + SOR_TY - 1) / SOR_TY, (d.np + SOR_KC - 1) / SOR_KC);
}

int sph_sor2_blocks(const SphDims& d) {
  const dim3 g = sor2_grid(d);
  return (int)(g.x * g.y * g.z);
}

cudaError_t launch_sph_gs(const SphDims& d, const SphTables& t, const double* rho, double fscale, double* g,
                          cudaStream_t s) {
  const long long nq = (long long)d.nr * d.nt;
  k_sph_gs<<<sph_grid(d), dim3(SBX, SBY), 0, s>>>(d, t.sor_tab + 5 * nq, rho, fscale, g);
  return cudaGetLastError();
}

cudaError_t launch_sph_sor2(const SphDims& d, const SphTables& t, double* x, const double* g, int colour,
                            double omega, const double* wc, double* wn, double* partials,
                            const DevState* st, cudaStream_t s) {
  if (wn != nullptr && (wc == nullptr || t.rj2 == nullptr)) return cudaErrorInvalidValue;
  const dim3 grid = sor2_grid(d), blk(SOR_TX, SOR_TY);
  if (colour == 1) {
    if (partials == nullptr) return cudaErrorInvalidValue;
    k_sph_sor2<1><<<grid, blk, 0, s>>>(d, t.sor_tab, x, g, colour, omega, wc, wn, t.rj2, partials, st);
  } else {
    k_sph_sor2<0><<<grid, blk, 0, s>>>(d, t.sor_tab, x, g, colour, omega, wc, wn, t.rj2, nullptr, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_sph_rednorm(const SphDims& d, const SphTables& t, const double* x, const double* g,
                               double* partials, const DevState* st, cudaStream_t s) {
  k_sph_sor2<2><<<sor2_grid(d), dim3(SOR_TX, SOR_TY), 0, s>>>(
      d, t.sor_tab, const_cast<double*>(x), g, 0, 1.0, nullptr, nullptr, nullptr, partials, st);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ BiCGSTAB kernels
// One iteration: v = L phat; alpha; s = r - alpha v, shat = B^-1 s; t = L shat;
// omega; x += alpha phat + omega shat, r = s - omega t; then either the
// recurrence residual stands, or (on a drop to REPLACE_DROP of its largest
// value since the last replacement, a claim of convergence, a breakdown or the
// end of the budget) r is replaced by the FP64 true residual b - L x and the
// stopping decision is taken on it; last the direction update (or restart).
// The iterate is updated group-wise: the increments accumulate in z (FP64) and
// are added to x only at a replacement, so x is rounded once per replacement
// (every rounding of x is amplified by the pole coefficients, up to ~1e11).
// The Krylov vectors are stored as T (double or float); x, the right-hand side
// f = fscale * rho and all dot products are FP64.

//   mode 0: partials {|b|^2, |b|^2} for b = f - L(boundary part of x)
//   mode 1: r = rhat = p = f - L x, phat = B^-1 r; partials {r.r, r.r}
//   mode 2 (only while st->replace is set): r = f - L x; partials
//           {r.r (FP64), rhat.r}
template <typename T>
__global__ void __launch_bounds__(SBX* SBY)
    k_bicg_resid(SphDims d, Tab<double> tb, const double* __restrict__ vol, int mode,
                 const double* __restrict__ rho, double fscale,
                 const double* __restrict__ x, T* __restrict__ r, T* __restrict__ rhat,
                 T* __restrict__ p, T* __restrict__ phat, double* __restrict__ partials,
                 const DevState* __restrict__ st) {
  if (mode == 2 && (st->done || !st->replace)) return;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  double s0 = 0.0, s1 = 0.0;
  if (i < d.nr && j < d.nt) {
    const long long c = d.at(i, j, k);
    // mode 0: the outer ghost enters through rad_p at i = nr-1 and a Dirichlet
    // inner ghost through rad_m at i = 0, nothing else.  f = fscale rho and
    // rv = f - L x are rounded separately, with explicitly rounded operations
    // that no contraction can merge: BiCGSTAB's step count on graded grids follows
    // every last bit of the true residual (one fused rounding here moved the
    // 32x16x32 test from 182 to 208 steps), and this is the oracle's order.
    double Lx;
    if (mode == 0) {
      Lx = __dmul_rn(tb.rad_p[i], i == d.nr - 1 ? x[c + 1] : 0.0);
      if (d.inner_ghost && i == 0) Lx = __dadd_rn(Lx, __dmul_rn(tb.rad_m[i], x[c - 1]));
    } else {
      Lx = sph_L<double, double>(d, tb, x, i, j, k, c);
    }
    const double rv = __dsub_rn(__dmul_rn(fscale, rho[c]), Lx);
    s0 = rv * rv;
    s1 = s0;
    if (sizeof(T) == 4 && mode != 0) {
      // refinement form: the inner solve's residual is V r (its Krylov process
      // restarts from it, so s1 is its squared norm); phat = (V D)^-1 V r = D^-1 r
      const double rsv = rv * vol[j * d.nr + i];
      s1 = rsv * rsv;
      r[c] = (T)rsv;
      if (mode == 1) {
        rhat[c] = (T)rsv;
        p[c] = (T)rsv;
        phat[c] = (T)(rv * tb.inv_diag[j * d.nr + i]);
      }
    } else if (mode == 1) {
      r[c] = (T)rv;
      rhat[c] = (T)rv;
      p[c] = (T)rv;
      phat[c] = (T)(rv * tb.inv_diag[j * d.nr + i]);
    } else if (mode == 2) {
      const T rs = (T)rv;
      r[c] = rs;
      s1 = (double)rs * (double)rhat[c];
    }
  }
  block_sum2(s0, s1, partials);
}

// The vector kernels of an iteration march a chunk of BKC phi planes per
// thread (block 32 r x 8 theta): the per-(r, theta) coefficients stay in
// registers, the phi neighbours slide along the chunk, and a block's partial
// dot products -- whose shuffle tree costs the FP64 pipe about ten instructions
// per thread -- are formed once per BKC nodes instead of once per node.  The
// arithmetic of every node is the one of sph_L.
static constexpr int BKC = 8;
static inline dim3 bk_grid(const SphDims& d) {
  return dim3((d.nr + SBX - 1) / SBX, (d.nt + SBY - 1) / SBY, (d.np + BKC - 1) / BKC);
}

// dst = L src; partials {dst.w1, dst.dst (with_tt)}
template <typename T>
__global__ void __launch_bounds__(SBX* SBY)
    k_bicg_apply(SphDims d, Tab<typename St<T>::C> tb, const T* __restrict__ src, T* __restrict__ dst,
                 const T* __restrict__ w1, int with_tt, double* __restrict__ partials,
                 const DevState* __restrict__ st) {
  using C = typename St<T>::C;
  if (st->done) return;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y;
  const int k0 = blockIdx.z * BKC, k1 = min(k0 + BKC, d.np);
  double s0 = 0.0, s1 = 0.0;
  if (i < d.nr && j < d.nt) {
    const C rp = tb.rad_p[i], rm = tb.rad_m[i], ir2 = tb.inv_r2[i];
    const C tp = tb.th_p[j], tm = tb.th_m[j], phc = tb.ph[j];
    C vs = (C)1;
    if constexpr (sizeof(C) == 4) vs = tb.vol[j * d.nr + i];
    const long long sy = d.sy(), sz = d.sz(), wrap = (long long)(d.np - 1) * sz;
    long long c = d.at(i, j, k0);
    C pkm = (C)(k0 == 0 ? src[c + wrap] : src[c - sz]);
    C pc = (C)src[c];
    for (int k = k0; k < k1; k++, c += sz) {
      const C pkp = (C)(k == d.np - 1 ? src[c - wrap] : src[c + sz]);
      const C pim = (C)(i == 0 && !d.inner_ghost ? src[c + 1] : src[c - 1]);
      const C pip = (C)src[c + 1];
      const C pjm = j == 0 ? pc : (C)src[c - sy];
      const C pjp = j == d.nt - 1 ? pc : (C)src[c + sy];
      C kk;
      if constexpr (sizeof(C) == 4) kk = (pkp - pc) + (pkm - pc);
      else kk = (pkp + pkm) - (C)2 * pc;
      const C ang = fma(tp, pjp - pc, fma(-tm, pc - pjm, phc * kk));
      C v = fma(rp, pip - pc, fma(-rm, pc - pim, ir2 * ang));
      if constexpr (sizeof(C) == 4) v *= vs;
      dst[c] = (T)v;
      const double vd = (double)v;
      s0 = fma(vd, (double)w1[c], s0);
      if (with_tt) s1 = fma(vd, vd, s1);
      pkm = pc;
      pc = pkp;
    }
  }
  if (with_tt) block_sum2(s0, s1, partials);
  else block_sum1(s0, partials);
}

// s = r - alpha v, shat = B^-1 s
template <typename T>
__global__ void __launch_bounds__(SBX* SBY)
    k_bicg_s(SphDims d, Tab<typename St<T>::C> tb, const T* __restrict__ r, const T* __restrict__ v,
             T* __restrict__ sv, T* __restrict__ shat, const DevState* __restrict__ st) {
  using C = typename St<T>::C;
  if (st->done) return;
  const C alpha = (C)st->alpha;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y;
  const int k0 = blockIdx.z * BKC, k1 = min(k0 + BKC, d.np);
  if (i >= d.nr || j >= d.nt) return;
  const C idg = tb.inv_diag[j * d.nr + i];
  const long long sz = d.sz();
  long long c = d.at(i, j, k0);
  for (int k = k0; k < k1; k++, c += sz) {
    const C s = fma(-alpha, (C)v[c], (C)r[c]);
    sv[c] = (T)s;
    shat[c] = (T)(s * idg);
  }
}

// z += alpha phat + omega shat (FP64 increments since the last replacement),
// r = s - omega t; partials {r.r, rhat.r}
template <typename T>
__global__ void __launch_bounds__(SBX* SBY)
    k_bicg_xr(SphDims d, double* __restrict__ z, T* __restrict__ r, const T* __restrict__ rhat,
              const T* __restrict__ phat, const T* __restrict__ sv, const T* __restrict__ shat,
              const T* __restrict__ tv, double* __restrict__ partials,
              const DevState* __restrict__ st) {
  using C = typename St<T>::C;
  if (st->done) return;
  const double alpha = st->alpha, omega = st->omega;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y;
  const int k0 = blockIdx.z * BKC, k1 = min(k0 + BKC, d.np);
  double s0 = 0.0, s1 = 0.0;
  if (i < d.nr && j < d.nt) {
    const long long sz = d.sz();
    long long c = d.at(i, j, k0);
    for (int k = k0; k < k1; k++, c += sz) {
      z[c] += fma(omega, (double)shat[c], alpha * (double)phat[c]);
      const C rv = fma(-(C)omega, (C)tv[c], (C)sv[c]);
      r[c] = (T)rv;
      const double rd = (double)rv;
      s0 = fma(rd, rd, s0);
      s1 = fma(rd, (double)rhat[c], s1);
    }
  }
  block_sum2(s0, s1, partials);
}

// Group-wise update at a replacement: x += z, z = 0 (refinement form: a
// discarded inner solve leaves x as it was).
__global__ void __launch_bounds__(SBX* SBY)
    k_bicg_fold(SphDims d, double* __restrict__ x, double* __restrict__ z,
                const DevState* __restrict__ st) {
  if (st->done || !st->replace) return;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y, k = blockIdx.z;
  if (i >= d.nr || j >= d.nt) return;
  const long long c = d.at(i, j, k);
  if (!st->discard) x[c] += z[c];
  z[c] = 0.0;
}

// p = r + beta (p - omega v), phat = B^-1 p; on a restart rhat = p = r.
template <typename T>
__global__ void __launch_bounds__(SBX* SBY)
    k_bicg_p(SphDims d, Tab<typename St<T>::C> tb, const T* __restrict__ r, T* __restrict__ rhat,
             T* __restrict__ p, const T* __restrict__ v, T* __restrict__ phat,
             const DevState* __restrict__ st) {
  using C = typename St<T>::C;
  if (st->done) return;
  const C beta = (C)st->beta, omega = (C)st->omega;
  const int restart = st->restart;
  const int i = blockIdx.x * SBX + threadIdx.x, j = blockIdx.y * SBY + threadIdx.y;
  const int k0 = blockIdx.z * BKC, k1 = min(k0 + BKC, d.np);
  if (i >= d.nr || j >= d.nt) return;
  const C idg = tb.inv_diag[j * d.nr + i];
  const long long sz = d.sz();
  long long c = d.at(i, j, k0);
  for (int k = k0; k < k1; k++, c += sz) {
    if (restart) {
      const T rv = r[c];
      rhat[c] = rv;
      p[c] = rv;
      phat[c] = (T)((C)rv * idg);
      continue;
    }
    const C pv = fma(beta, fma(-omega, (C)v[c], (C)p[c]), (C)r[c]);
    p[c] = (T)pv;
    phat[c] = (T)(pv * idg);
  }
}

// refinement form: no iteration cap on an inner FP32 solve until one overflows
static constexpr int kNoCap = 1 << 30;

__device__ __forceinline__ void bicg_set_loop(const DevState* st, unsigned long long cond, int chunk) {
  if (chunk > 0) {
    const unsigned int more = (st->done == DONE_NO && st->iter < st->chunk_end) ? 1u : 0u;
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond, more);
  }
}

// Direction update from the current residual (r.r = rr, rhat.r = rho_new):
// beta as usual, or a restart rhat = p = r after a breakdown of alpha or omega
// or an exactly vanishing rhat.r.
__device__ __forceinline__ void bicg_direction(DevState* st, double rr, double rho_new) {
  if (st->broke || rho_new == 0.0) {
    st->restart = 1;
    st->rho = rr;
    st->beta = 0.0;
  } else {
    st->beta = (rho_new / st->rho) * (st->alpha / st->omega);
    st->rho = rho_new;
  }
  st->broke = 0;
}

__device__ __forceinline__ void sum_partials2(const double* __restrict__ partials, int nblk,
                                              double* sh, double (&v)[2]) {
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
    a += partials[2 * q];
    b += partials[2 * q + 1];
  }
  v[0] = a;
  v[1] = b;
  block_sum<2>(v, sh);
}

// which: 0 alpha; 2 omega; 3 recurrence residual (direction update, or a
// replacement request that k_bicg_replace_finish completes).
__global__ void k_bicg_scalar(const double* __restrict__ partials, int nblk, int which,
                              DevState* __restrict__ st, unsigned long long cond, int chunk) {
  __shared__ double sh[64];
  if (st->done) {
    if (which == 3 && threadIdx.x == 0) bicg_set_loop(st, cond, chunk);
    return;
  }
  double v[2];
  sum_partials2(partials, nblk, sh, v);
  if (threadIdx.x != 0) return;
  if (which == 0) {
    st->restart = 0;
    const double al = st->rho / v[0];
    st->broke = isfinite(al) ? 0 : 1;
    st->alpha = isfinite(al) ? al : 0.0;
  } else if (which == 2) {
    st->ts = v[0];
    st->tt = v[1];
    const double om = v[0] / v[1];
    if (isfinite(om) && om != 0.0) {
      st->omega = om;
    } else {
      st->omega = 0.0;
      st->broke = 1;
    }
  } else {
    st->iter += 1;
    const double rn = sqrt(v[0]);
    // refinement form: an inner solve whose FP32 recursion overflowed (a
    // non-finite residual: one of BiCGSTAB's excursions on graded grids grew
    // past the FP32 range) is discarded -- its increments are dropped and x is
    // kept -- and the next inner solve from the same x is capped at half as
    // many iterations, so it stops before that excursion; a successful inner
    // solve lifts the cap again.
    bool inner_end = false;
    if (st->restart_on_replace) {
      const bool bad = !isfinite(rn);
      inner_end = bad || st->iter - st->iter_repl >= st->inner_cap;
      st->discard = bad ? 1 : 0;
    }
    // (the refinement form's recursive norm is of V r; only its replaced, FP64
    // true residual is compared with the tolerance)
    const bool claims = !st->restart_on_replace && rn / st->ref <= st->tol;
    if (!isfinite(rn) || st->broke || rn <= st->replace_drop * st->rmax || claims ||
        st->iter >= st->max_iter || inner_end) {
      st->replace = 1;   // k_bicg_replace_finish decides and sets the loop
      return;
    }
    st->rmax = fmax(st->rmax, rn);
    st->rr = v[0];
    st->rel = rn / st->ref;
    bicg_direction(st, v[0], v[1]);
    bicg_set_loop(st, cond, chunk);
  }
}

// After a residual replacement: stop on the true residual, else continue the
// search direction from it.
__global__ void k_bicg_replace_finish(const double* __restrict__ partials, int nblk,
                                      DevState* __restrict__ st, unsigned long long cond, int chunk) {
  __shared__ double sh[64];
  if (st->done || !st->replace) return;   // the loop condition is already set
  double v[2];
  sum_partials2(partials, nblk, sh, v);
  if (threadIdx.x != 0) return;
  st->replace = 0;
  st->inner_cycles += 1;
  if (st->restart_on_replace)
    st->inner_cap = st->discard ? max(8, (st->iter - st->iter_repl) / 2) : kNoCap;
  st->discard = 0;
  st->iter_repl = st->iter;
  const double rn = sqrt(v[0]);
  st->rmax = st->restart_on_replace ? sqrt(v[1]) : rn;   // refinement form: ||V r||
  st->rr = v[0];
  st->rel = rn / st->ref;
  if (st->rel <= st->tol) st->done = DONE_CONVERGED;
  else if (!isfinite(rn)) st->done = DONE_DIVERGED;
  else if (st->iter >= st->max_iter) st->done = DONE_MAXITER;
  else {
    // refinement form (FP32 Krylov vectors): a new Krylov process starts from
    // the FP64 true residual
    if (st->restart_on_replace) {
      st->broke = 1;
      bicg_direction(st, v[1], v[1]);   // rho = ||V r||^2 of the new process
    } else {
      bicg_direction(st, v[0], v[1]);
    }
  }
  bicg_set_loop(st, cond, chunk);
}

__global__ void k_bicg_start(const double* __restrict__ partials, int nblk, int mode,
                             DevState* __restrict__ st, double replace_drop, int restart_on_replace) {
  __shared__ double sh[64];
  double v[2];
  sum_partials2(partials, nblk, sh, v);
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    const double ref = sqrt(v[0]);
    st->ref = ref > 0.0 ? ref : 1.0;
    st->amax = ref;
    return;
  }
  st->rr = v[0];
  st->rho = v[1];
  st->rmax = restart_on_replace ? sqrt(v[1]) : sqrt(v[0]);
  st->replace_drop = replace_drop;
  st->restart_on_replace = restart_on_replace;
  st->iter_repl = 0;
  st->discard = 0;
  st->inner_cap = kNoCap;
  st->iter = 0;
  st->broke = 0;
  st->restart = 0;
  st->replace = 0;
  const double rel = sqrt(v[0]) / st->ref;
  st->rel = rel;
  st->rel0 = rel;
  st->done = rel <= st->tol ? DONE_CONVERGED : (st->max_iter <= 0 ? DONE_MAXITER : DONE_NO);
  if (!isfinite(rel)) st->done = DONE_DIVERGED;
}

cudaError_t launch_bicg_resid(const SphDims& d, const SphTables& t, int dt, int mode,
                              const double* rho, double fscale, const double* x, void* r,
                              void* rhat, void* p, void* phat, double* partials, int* nblk,
                              cudaStream_t s) {
  const dim3 g = sph_grid(d), b(SBX, SBY);
  if (nblk) *nblk = g.x * g.y * g.z;
  if (dt == DT_F64)
    k_bicg_resid<double><<<g, b, 0, s>>>(d, tab_of<double>(t), t.vol, mode, rho, fscale, x, (double*)r,
                                         (double*)rhat, (double*)p, (double*)phat, partials, nullptr);
  else
    k_bicg_resid<float><<<g, b, 0, s>>>(d, tab_of<double>(t), t.vol, mode, rho, fscale, x, (float*)r,
                                        (float*)rhat, (float*)p, (float*)phat, partials, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_bicg_start(const double* partials, int nblk, int mode, DevState* st,
                              cudaStream_t s, double replace_drop, int restart_on_replace) {
  k_bicg_start<<<1, 256, 0, s>>>(partials, nblk, mode, st, replace_drop, restart_on_replace);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t iter_t(const SphDims& d, const SphTables& t, const double* rho, double fscale,
                          double* x, double* z, void* r, void* rhat, void* p, void* phat, void* v,
                          void* sv, void* shat, void* tv, double* partials, DevState* st,
                          cudaStream_t s, unsigned long long cond, int chunk) {
  using C = typename St<T>::C;
  const Tab<C> tb = tab_of<C>(t);
  const dim3 g = sph_grid(d), gk = bk_grid(d), b(SBX, SBY);
  const int nblk = g.x * g.y * g.z, nblk_k = gk.x * gk.y * gk.z;
  k_bicg_apply<T><<<gk, b, 0, s>>>(d, tb, (const T*)phat, (T*)v, (const T*)rhat, 0, partials, st);
  k_bicg_scalar<<<1, 1024, 0, s>>>(partials, nblk_k, 0, st, 0ull, 0);
  k_bicg_s<T><<<gk, b, 0, s>>>(d, tb, (const T*)r, (const T*)v, (T*)sv, (T*)shat, st);
  k_bicg_apply<T><<<gk, b, 0, s>>>(d, tb, (const T*)shat, (T*)tv, (const T*)sv, 1, partials, st);
  k_bicg_scalar<<<1, 1024, 0, s>>>(partials, nblk_k, 2, st, 0ull, 0);
  k_bicg_xr<T><<<gk, b, 0, s>>>(d, z, (T*)r, (const T*)rhat, (const T*)phat, (const T*)sv,
                                (const T*)shat, (const T*)tv, partials, st);
  k_bicg_scalar<<<1, 1024, 0, s>>>(partials, nblk_k, 3, st, cond, chunk);
  k_bicg_fold<<<g, b, 0, s>>>(d, x, z, st);
  k_bicg_resid<T><<<g, b, 0, s>>>(d, tab_of<double>(t), t.vol, 2, rho, fscale, x, (T*)r, (T*)rhat,
                                  nullptr, nullptr, partials, st);
  k_bicg_replace_finish<<<1, 1024, 0, s>>>(partials, nblk, st, cond, chunk);
  k_bicg_p<T><<<gk, b, 0, s>>>(d, tb, (const T*)r, (T*)rhat, (T*)p, (const T*)v, (T*)phat, st);
  return cudaGetLastError();
}

cudaError_t launch_bicg_iter(const SphDims& d, const SphTables& t, int dt, const double* rho,
                             double fscale, double* x, double* z, void* r, void* rhat, void* p,
                             void* phat, void* v, void* sv, void* shat, void* tv, double* partials,
                             DevState* st, cudaStream_t s, unsigned long long cond, int chunk) {
  if (dt == DT_F64)
    return iter_t<double>(d, t, rho, fscale, x, z, r, rhat, p, phat, v, sv, shat, tv, partials, st, s, cond, chunk);
  return iter_t<float>(d, t, rho, fscale, x, z, r, rhat, p, phat, v, sv, shat, tv, partials, st, s, cond, chunk);
}

int bicg_iter_kernels(int) { return 11; }

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

// Eq. outer_expansion on the outer ghost shell (radial factors rg^-(l+1)), or
// (inner) Eq. inner_expansion on the inner ghost shell (factors rg^l)
__global__ void __launch_bounds__(256)
    k_sph_face(SphDims d, int L, double G, double rg, const double* __restrict__ q,
               const double* __restrict__ Pn, const double* __restrict__ cosT,
               const double* __restrict__ sinT, double* __restrict__ phi, int inner) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= d.nt * d.np) return;
  const int j = id % d.nt, k = id / d.nt;
  double acc = 0.0, rl = inner ? 1.0 : 1.0 / rg;
  const double ir = inner ? rg : 1.0 / rg;
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
  phi[d.at(inner ? -1 : d.nr, j, k)] = -G * acc;
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
  if (t.q_in != nullptr)   // the inner moments share the phi-Fourier and theta passes
    k_sph_moments<<<(L + 1) * (L + 1), 256, 0, s>>>(d, L, t.Pn, t.sinth, t.Rw_in, t.Fc, t.Fs, t.q_in);
  return cudaGetLastError();
}

cudaError_t launch_sph_face_inner(const SphDims& d, const SphTables& t, double G, double* phi,
                                  cudaStream_t s) {
  if (t.q_in == nullptr) return cudaErrorInvalidValue;
  const int n = d.nt * d.np;
  k_sph_face<<<(n + 255) / 256, 256, 0, s>>>(d, t.lmax, G, t.r_ghost_in, t.q_in, t.Pn, t.cosT, t.sinT, phi, 1);
  return cudaGetLastError();
}

cudaError_t launch_sph_face(const SphDims& d, const SphTables& t, double G, double* phi,
                            cudaStream_t s) {
  const int n = d.nt * d.np;
  k_sph_face<<<(n + 255) / 256, 256, 0, s>>>(d, t.lmax, G, t.r_ghost, t.q, t.Pn, t.cosT, t.sinT, phi, 0);
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
                             int lmax, SphTables* t, bool inner_multipole) {
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
  {
    // cell volumes r_i^2 dr_i sin(theta_j) (dtheta dphi dropped), normalised to
    // at most 1: the row scaling that makes the flux form symmetric
    std::vector<double> vol((size_t)nr * nt), idv((size_t)nr * nt);
    double vmax = 0.0;
    for (int j = 0; j < nt; j++)
      for (int i = 0; i < nr; i++) {
        const double ri = re[i + 1], dr = 0.5 * (re[i + 2] - re[i]);
        vol[(size_t)j * nr + i] = ri * ri * dr * std::sin(th[j]);
        vmax = std::max(vmax, vol[(size_t)j * nr + i]);
      }
    for (size_t q = 0; q < vol.size(); q++) {
      vol[q] /= vmax;
      idv[q] = idg[q] / vol[q];
    }
    if ((e = upload(&t->vol, vol, &t->bytes)) != cudaSuccess) return e;
    if ((e = upload(&t->volf, to_f(vol), &t->bytes)) != cudaSuccess) return e;
    if ((e = upload(&t->inv_diag_vf, to_f(idv), &t->bytes)) != cudaSuccess) return e;
  }
  // Eq. local_rjac: rJ at (theta_j, r_i) from the radial width of the flux form,
  // r_i dtheta and r_i sin(theta_j) dphi; stored squared for the SOR weights
  std::vector<double> rjsq((size_t)nr * nt);
  const double cr = std::cos(M_PI / nr), ct = std::cos(M_PI / nt), cp = std::cos(M_PI / np);
  for (int j = 0; j < nt; j++)
    for (int i = 0; i < nr; i++) {
      const double ri = re[i + 1], dr = 0.5 * (re[i + 2] - re[i]);
      const double wr = 1.0 / (dr * dr);
      const double wt = 1.0 / ((ri * dth) * (ri * dth));
      const double wp = 1.0 / ((ri * sth[j] * dph) * (ri * sth[j] * dph));
      const double rj = (cr * wr + ct * wt + cp * wp) / (wr + wt + wp);
      rjsq[(size_t)j * nr + i] = rj * rj;
    }
  if ((e = upload(&t->rj2, rjsq, &t->bytes)) != cudaSuccess) return e;
  {
    const size_t nq = (size_t)nr * nt;
    std::vector<double> sb(6 * nq);
    for (int j = 0; j < nt; j++)
      for (int i = 0; i < nr; i++) {
        const size_t q = (size_t)j * nr + i;
        const double ac = rp[i] + rm[i] + ir2[i] * (tp[j] + tm[j] + 2.0 * pp[j]);
        sb[0 * nq + q] = rp[i] / ac;
        sb[1 * nq + q] = rm[i] / ac;
        sb[2 * nq + q] = ir2[i] * tp[j] / ac;
        sb[3 * nq + q] = ir2[i] * tm[j] / ac;
        sb[4 * nq + q] = ir2[i] * pp[j] / ac;
        sb[5 * nq + q] = ac;
      }
    if ((e = upload(&t->sor_tab, sb, &t->bytes)) != cudaSuccess) return e;
  }
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
    if (inner_multipole) {
      // Eq. inner_multipole: r'^-(l+1) times the volume factor r'^2 dr dtheta dphi
      std::vector<double> Rwi((size_t)W * nr);
      for (int i = 0; i < nr; i++) {
        const double dr = 0.5 * (re[i + 2] - re[i]);
        double rl = r[i];
        for (int l = 0; l < W; l++) {
          Rwi[(size_t)l * nr + i] = rl * dr * dth * dph;
          rl /= r[i];
        }
      }
      if ((e = upload(&t->Rw_in, Rwi, &t->bytes)) != cudaSuccess) return e;
      if ((e = cudaMalloc(&t->q_in, (size_t)W * W * sizeof(double))) != cudaSuccess) return e;
      t->bytes += (size_t)W * W * sizeof(double);
      t->r_ghost_in = re[0];
    }
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
                  t->cosT, t->sinT, t->Pn, t->Rw, t->sinth, t->Fc, t->Fs, t->q, t->rj2, t->Rw_in, t->q_in,
                  t->sor_tab, t->vol, t->volf, t->inv_diag_vf};
  for (void* p : ptrs) cudaFree(p);
  *t = SphTables();
}

}  // namespace ps
