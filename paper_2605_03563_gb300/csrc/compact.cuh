// Compact radius-one stencils, SPAI smoothing and Galerkin coarse operators
// (Sec. 2.1.3), FP64, on radius-one (order 2) level layouts.
//
// An isotropic 27-point stencil is given by its weights per offset class:
// w[0] centre, w[1] the 6 faces, w[2] the 12 edges, w[3] the 8 corners, in
// absolute units (already divided by h^2 where the operator carries it).
#pragma once
#include "ps_common.cuh"

namespace ps {

struct W27 {
  double w[4];
};

// Compact L_h of order 2, 4, 6 in units of 1/h^2, and the right-hand side R_h.
W27 compact_lhs(int order, double h);
// Galerkin coarse operator R A P (full weighting R, trilinear P = 8 R^T) of an
// isotropic 27-point A: the coarse stencil is again isotropic with radius one.
W27 galerkin27(const W27& fine);

// r = b - A u on the interior (FP64 arithmetic); with partials, per-block
// {sum r^2, 0} (c27_blocks(d) blocks).
cudaError_t launch_c27_resid(const Dims& d, const W27& A, const double* u, const double* b, double* r,
                             double* partials, const DevState* st, cudaStream_t s);
// the same with r stored as dt_r (DT_F64 or DT_F32: the refinement's outer
// residual, rounded to FP32 on the integer pipe)
cudaError_t launch_c27_resid_dt(const Dims& d, const W27& A, const double* u, const double* b, int dt_r, void* r,
                                double* partials, const DevState* st, cudaStream_t s);
int c27_blocks(const Dims& d);
// Initial residual of a compact solve: r = b - A u (stored FP64 or FP32 per
// dt_r) with per-block partials {sum r^2, 0} at partials[0 .. 2 nb) and the
// reference residual b - A u0 (u0: boundary data of u only) as partials at
// partials[2 nb .. 4 nb), nb = c27_blocks(d), in one pass.
cudaError_t launch_c27_init(const Dims& d, const W27& A, const double* u, const double* b, int dt_r, void* r,
                            double* partials, cudaStream_t s);
// u -= omega M r on the interior (Eq. richardson for A = -L_h with M of Eq. Smoother)
cudaError_t launch_c27_spai(const Dims& d, const W27& M, double omega, const double* r, double* u,
                            const DevState* st, cudaStream_t s);
// b = R_h (fscale rho) on the interior; rho in the caller's dense layout du
cudaError_t launch_c27_rhs(const Dims& d, const Dims& du, int order, const double* rho, double fscale,
                           double* b, cudaStream_t s);
// coarsest level: CG on -A u = -b from u = 0 in one CTA, to ||r|| <= tol ||b||
// or as many iterations as unknowns; u receives the result
cudaError_t launch_c27_coarse_cg(const Dims& d, const W27& A, const double* b, double* u, double tol,
                                 const DevState* st, cudaStream_t s);
size_t c27_coarse_smem(const Dims& d);

// FP32 passes of the refinement's inner cycles on level layouts with 16-byte
// aligned rows (TMA-staged; a stage wait that times out sets *fault).
// One SPAI smoothing step u' = u - omega M (b - A u) in one pass, written to
// dst (dst != u; u's boundary nodes read as the boundary data, dst's boundary
// nodes are left as they are).
cudaError_t launch_c27_smooth(const Dims& d, const W27& A, const W27& M, double omega, const float* u,
                              const float* b, float* dst, const DevState* st, int* fault, cudaStream_t s);
// r = b - A u on the interior (the residual before a restriction; r != u)
cudaError_t launch_c27_resid_f32(const Dims& d, const W27& A, const float* u, const float* b, float* r,
                                 const DevState* st, int* fault, cudaStream_t s);
// coarsest CG in FP64 arithmetic on FP32 or FP64 storage
cudaError_t launch_c27_coarse_cg_dt(const Dims& d, const W27& A, int dt, const void* b, void* u, double tol,
                                    const DevState* st, cudaStream_t s);

}  // namespace ps
