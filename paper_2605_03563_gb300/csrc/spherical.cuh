// Spherical-grid operator, BiCGSTAB kernels and multipole (Eq. 2, Sec. 2.1.2, Sec. 2.2).
#pragma once
#include <vector>

#include "multipole.cuh"
#include "ps_common.cuh"

namespace ps {

// Ghosted layout (Nr+2, Ntheta+2, Nphi+2), r fastest; node (i,j,k) at
// ((k+1)*(nt+2) + (j+1))*(nr+2) + (i+1).
struct SphDims {
  int nr, nt, np;
  int inner_ghost;   // 0: Neumann mirror P_{-1} = P_1; 1: the inner ghost shell holds Dirichlet data
  __host__ __device__ long long sy() const { return nr + 2; }
  __host__ __device__ long long sz() const { return (long long)(nr + 2) * (nt + 2); }
  __host__ __device__ long long size() const { return sz() * (np + 2); }
  __host__ __device__ long long at(int i, int j, int k) const {
    return ((long long)(k + 1) * (nt + 2) + (j + 1)) * (nr + 2) + (i + 1);
  }
};

// 1-D coefficient tables of the flux-form operator (device, FP64):
//   rad_p[i], rad_m[i], inv_r2[i]  (Nr), th_p[j], th_m[j], ph[j] (Ntheta),
//   inv_diag[j*Nr+i] (Nr*Ntheta).
struct SphTables {
  double *rad_p = nullptr, *rad_m = nullptr, *inv_r2 = nullptr;
  double *th_p = nullptr, *th_m = nullptr, *ph = nullptr;
  double* inv_diag = nullptr;
  float *rad_pf = nullptr, *rad_mf = nullptr, *inv_r2f = nullptr;   // FP32 copies
  float *th_pf = nullptr, *th_mf = nullptr, *phf = nullptr, *inv_diagf = nullptr;
  // multipole tables
  int lmax = -1;
  double* cosT = nullptr;   // [(L+1) * Nphi]
  double* sinT = nullptr;
  double* Pn = nullptr;     // [(L+1)^2 (m>=0 packed as l*(L+1)+m) * Ntheta]
  double* Rw = nullptr;     // [(L+1) * Nr]: r_i^(l+2) dr_i dtheta dphi
  double* sinth = nullptr;  // [Ntheta]
  double* Fc = nullptr;     // [(L+1) * Ntheta * Nr]
  double* Fs = nullptr;
  double* q = nullptr;      // [(L+1)^2]
  double r_ghost = 0.0;     // outer ghost radius
  // SOR: rJ^2 of Eq. local_rjac per (theta_j, r_i) [Ntheta * Nr]
  double* rj2 = nullptr;
  // inner expansion (Eqs. inner_multipole / inner_expansion): radial weights
  // r_i^(1-l) dr_i dtheta dphi [(L+1) * Nr], moments qbar [(L+1)^2], ghost radius
  double* Rw_in = nullptr;
  double* q_in = nullptr;
  double r_ghost_in = 0.0;
  // SOR in the scaled Gauss-Seidel form, per (theta_j, r_i) [6][Ntheta * Nr]:
  // b_ip, b_im, b_jp, b_jm, b_k = the neighbour coefficients of L divided by
  // a_c = -diag(L) > 0, and a_c itself (x_GS = sum b x_nb + g, g = -f / a_c,
  // r = f - L x = a_c (x - x_GS))
  double* sor_tab = nullptr;
  // refinement form (FP32 inner solves on V L e = V r): cell volumes V per
  // (theta_j, r_i) normalised to at most 1 (FP64 and FP32) and 1 / (V diag(L)) (FP32)
  double* vol = nullptr;
  float* volf = nullptr;
  float* inv_diag_vf = nullptr;
  size_t bytes = 0;
};

cudaError_t sph_tables_build(const SphDims& d, const double* r, const double* th, const double* ph,
                             int lmax, SphTables* t, bool inner_multipole = false);
void sph_tables_free(SphTables* t);

// out = L phi on unknown nodes (phi's outer ghost as given, mirror + periodic by index)
cudaError_t launch_sph_apply(const SphDims& d, const SphTables& t, const double* phi, double* out,
                             cudaStream_t s);

// ---- BiCGSTAB (Krylov vectors stored as T = double or float; x, the
// right-hand side f = fscale * rho and every dot product in FP64)
// mode 0: ref norm of b = f - L(boundary part of x); mode 1: r = f - L x,
// rhat = p = r, phat = B^-1 r (FP64 arithmetic, stored as T).
cudaError_t launch_bicg_resid(const SphDims& d, const SphTables& t, int dt, int mode,
                              const double* rho, double fscale, const double* x, void* r,
                              void* rhat, void* p, void* phat, double* partials, int* nblk,
                              cudaStream_t s);
// One iteration (bicg_iter_kernels(dt) kernels).  The FP64 true residual
// replaces the recurrence one whenever the latter has dropped a hundredfold
// below its largest value since the last replacement or claims convergence,
// and every stopping decision is taken on a replaced residual.  With chunk > 0
// it runs inside a CUDA-graph while loop whose condition the last scalar
// kernel sets.
// x is the FP64 iterate, z (FP64, zero at the start) accumulates its
// increments between replacements (group-wise update).
cudaError_t launch_bicg_iter(const SphDims& d, const SphTables& t, int dt, const double* rho,
                             double fscale, double* x, double* z, void* r, void* rhat, void* p,
                             void* phat, void* v, void* sv, void* shat, void* tv, double* partials,
                             DevState* st, cudaStream_t s, unsigned long long cond = 0,
                             int chunk = 0);
int bicg_iter_kernels(int dt);
// scalar finisher for the reference / initial residual (mode 0/1)
cudaError_t launch_bicg_start(const double* partials, int nblk, int mode, DevState* st,
                              cudaStream_t s, double replace_drop = 0.01, int restart_on_replace = 0);

// ---- red-black SOR (Sec. 2.1.1) on the spherical grid, FP64.
// One colour pass: nodes with (i + j + k) mod 2 == colour take
// x += w (fscale rho - L x) * inv_diag; w = omega, or wc[j*Nr + i] when wc is
// given.  With wn given as well, the pass also writes the next pass's weights
// wn = 1 / (1 - rJ^2 wc / 4) (Eq. omega_n per node).  Skipped once st->done.
cudaError_t launch_sph_sor(const SphDims& d, const SphTables& t, double* x, const double* rho,
                           double fscale, int colour, double omega, const double* wc, double* wn,
                           const DevState* st, cudaStream_t s);
// Red-black SOR step in the scaled form (tables sor_tab, g = -fscale rho / a_c
// from launch_sph_gs): colour pass `colour` (0 red, then 1 black), thread per
// (i pair, j) marching a chunk of phi planes.  The black pass (partials
// required) also writes the per-block partials of sum r^2 over the black nodes
// after their update (partials[0 .. nblk)); launch_sph_rednorm then adds the
// red nodes' residuals (partials[nblk .. 2 nblk)).  Weights as launch_sph_sor.
cudaError_t launch_sph_gs(const SphDims& d, const SphTables& t, const double* rho, double fscale,
                          double* g, cudaStream_t s);
cudaError_t launch_sph_sor2(const SphDims& d, const SphTables& t, double* x, const double* g, int colour,
                            double omega, const double* wc, double* wn, double* partials,
                            const DevState* st, cudaStream_t s);
cudaError_t launch_sph_rednorm(const SphDims& d, const SphTables& t, const double* x, const double* g,
                               double* partials, const DevState* st, cudaStream_t s);
int sph_sor2_blocks(const SphDims& d);
// partials {sum r^2, 0} of r = fscale rho - L x over the unknown nodes; *nblk = blocks
cudaError_t launch_sph_resnorm(const SphDims& d, const SphTables& t, const double* x,
                               const double* rho, double fscale, double* partials, int* nblk,
                               cudaStream_t s);
int sph_resnorm_blocks(const SphDims& d);
// w[j*Nr + i] = omega_1 (chebyshev) or omega_opt (Eq. 3) of the local rJ
cudaError_t launch_sph_sor_weights(const SphDims& d, const SphTables& t, int chebyshev, double* w,
                                   cudaStream_t s);

// multipole: q <- moments of rho (unknown nodes, dV = r^2 sin t dr dt dp);
// outer ghost of phi <- expansion at r_ghost
cudaError_t launch_sph_moments(const SphDims& d, const SphTables& t, const double* rho,
                               cudaStream_t s);
cudaError_t launch_sph_face(const SphDims& d, const SphTables& t, double G, double* phi,
                            cudaStream_t s);
// inner ghost shell of phi <- Eq. inner_expansion at r_ghost_in (after launch_sph_moments
// with the inner tables, which then also forms qbar)
cudaError_t launch_sph_face_inner(const SphDims& d, const SphTables& t, double G, double* phi,
                                  cudaStream_t s);

}  // namespace ps
