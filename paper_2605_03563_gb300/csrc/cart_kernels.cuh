// Host-side launchers of the Cartesian stencil kernels (cart_kernels.cu).
#pragma once
#include "ps_common.cuh"

namespace ps {

enum DType { DT_F64 = 0, DT_F32 = 1, DT_BF16 = 2 };

template <typename C>
Coef<C> make_coef(const Dims& d, const double h[3], int order);

// Which reduction a delta pass produces.
enum { RED_NONE = 0, RED_SUM2 = 1, RED_SUM2_MAX = 2 };

struct LaunchCfg {
  int nblocks;   // number of reduction partials the launch writes
};

// delta = phi_GS - phi on interior nodes (scaled residual, r = -d delta).
//   phi/fs: storage dtype `din`; out (optional): storage dtype `dout`, scaled by out_scale.
//   zero_interior: treat interior phi as zero (reference norm).
//   partials (optional): per block {sum delta^2, max |delta|}.
// Returns the number of blocks (partials written) via cfg.
cudaError_t launch_delta(const Dims& d, int order, const double h[3], int din, const void* phi,
                         const void* fs, int dout, void* out, double out_scale, bool zero_interior,
                         double* partials, LaunchCfg* cfg, cudaStream_t s);

// As launch_delta, storing delta * st->scale_next (iterative refinement).
cudaError_t launch_delta_st(const Dims& d, int order, const double h[3], int din, const void* phi,
                            const void* fs, int dout, void* out, const DevState* st,
                            double* partials, cudaStream_t s);

// delta = phi_GS - phi right after a complete omega = 1 colour sweep of phi: the
// last colour's delta is exactly zero (stored without evaluation), the other
// colours are evaluated.  Storage pairs (din, dout): F64/F64, F32/F32.  (With
// BF16 storage the last colour keeps its rounding error; use launch_delta.)
cudaError_t launch_delta_after_sweep(const Dims& d, int order, const double h[3], int din, const void* phi,
                                     const void* fs, int dout, void* out, cudaStream_t s);

// One colour pass of the multicolour GS/SOR sweep (skipped once st->done, if st given).
// With wtab (wlen >= 1 entries, st required) the pass's weight is
// wtab[min(ncolours * st->iter + colour, wlen - 1)] instead of omega.
cudaError_t launch_sweep_colour(const Dims& d, int order, const double h[3], int dt, void* phi,
                                const void* fs, int colour, double omega, const DevState* st,
                                cudaStream_t s, const double* wtab = nullptr, int wlen = 0);

// fs = factor * f on interior nodes, both of storage dt
cudaError_t launch_scale_rhs_any(const Dims& d, double factor, int dt, const void* f, void* fs,
                                 cudaStream_t s);

// FP64 13-point residual passes on equal spacings along (j, k) anti-diagonals
// (every delta equal to launch_delta's bit for bit; reductions in another
// order).  mode 0: partials {sum of delta^2 over colours 0 and 1, 0} (the norm
// after a sweep); 1: delta of colours 0 and 1 into out (FP64), zero on colour 2;
// 2: partials {sum of delta^2 over every node, 0}, and with st the initial
// residual pass, which writes nothing when st->guess_nonzero == 0 (finisher
// mode 4); 3: the refinement pass of launch_delta_st (out FP32 or BF16 scaled
// by st->scale_next, FP32 sum and max).  nblocks: the partials count,
// delta_diag13_blocks(d).
int delta_diag13_blocks(const Dims& d);
cudaError_t launch_delta_diag13(const Dims& d, const double h[3], int mode, const double* phi, const double* fs,
                                int dout, void* out, const DevState* st, double* partials, int* nblocks,
                                cudaStream_t s);

// Lagged convergence check of FP64 7-point V-cycles on equal spacings: the
// first colour pass (colour 0, omega = 1) of the next V-cycle; with norm it
// stores the old values of its nodes in save (node index p at save[p / 2]; the
// row pitch and plane stride of d must be even) and writes
// partials {sum of (x_GS - x_old)^2, 0} (nblocks blocks, at most
// delta_colours_partials(d, 2)); without norm it is the plain pass and marks
// st->lag_pending.  Skipped once st->done.
cudaError_t launch_sweep_lag(const Dims& d, const double h[3], double* phi, const double* fs, double* save,
                             bool norm, DevState* st, double* partials, int* nblocks, cudaStream_t s);
// phi <- save on the colour-0 nodes when st->lag_pending (undoes the last lagged pass).
cudaError_t launch_restore_colour0(const Dims& d, double* phi, const double* save, const DevState* st,
                                   cudaStream_t s);

// Set-up copy of the initial guess (same logical extents, dst pitch >= src
// pitch) that sets st->guess_nonzero when an interior node is nonzero.
cudaError_t launch_copy_guess(const Dims& dd, const Dims& sd, const double* src, double* dst, DevState* st,
                              cudaStream_t s);

// FP64 set-up pass: fs = factor * rho on interior nodes (rho in the layout du,
// fs in d: same logical extents) and the partials {sum, max} of the reference
// norm ||f - A phi0|| with every interior value of phi (layout du) read as
// zero (only the boundary data enter), per block of point_grid(d)
// (cart_partials_count blocks); the values equal launch_delta's with
// zero_interior up to the order in which the boundary terms are added.
cudaError_t launch_scale_rhs_ref(const Dims& d, const Dims& du, int order, const double h[3], double factor,
                                 const double* rho, const double* phi, double* fs, double* partials,
                                 cudaStream_t s);

// FP64 residual pass of the 7-point stencil on equal spacings along (j, k)
// diagonals (every delta equal to launch_delta's / launch_delta_st's bit for
// bit; the reductions run in another order).  out == NULL: partials {sum of
// delta^2, 0}; otherwise the refinement pass of launch_delta_st (out FP32 or
// BF16, scaled by st->scale_next, FP32 sum and max of the scaled values).
// Returns the block count in nblocks (at most delta_colours_partials(d, 2)).
// initial (st required): the solve's initial residual; when st->guess_nonzero
// == 0 the plain pass writes nothing (finisher mode 4) and the refinement pass
// takes its deltas from fs and the ghost values alone.
cudaError_t launch_delta_diag(const Dims& d, const double h[3], const double* phi, const double* fs, int dout,
                              void* out, const DevState* st, bool initial, double* partials, int* nblocks,
                              cudaStream_t s);

// fs_coarse = factor * R(delta_fine)  (scaled coarse right-hand side); coarse = layout of fs_c
cudaError_t launch_restrict(const Dims& fine, const Dims& coarse, int dt_f, const void* delta_f, int dt_c,
                            void* fs_c, double factor, cudaStream_t s);

// The same for a 7-point residual that is exactly zero on the black nodes
// ((i+j+k) odd), as launch_delta_after_sweep leaves it for order 2: the zero
// terms are dropped (9 arithmetic instructions per coarse node instead of 19);
// equal to launch_restrict bit for bit up to the sign of zero sums.  dt_f is
// FP64 or FP32.
cudaError_t launch_restrict_red(const Dims& fine, const Dims& coarse, int dt_f, const void* delta_f, int dt_c,
                                void* fs_c, double factor, cudaStream_t s);

// phi_fine += P e_coarse; coarse = layout of e_c
cudaError_t launch_prolong(const Dims& fine, const Dims& coarse, int dt_c, const void* e_c, int dt_f, void* phi_f,
                           cudaStream_t s);

// fs = -(4 pi G / d) rho on interior nodes (rho FP64 in layout du, fs in layout d)
cudaError_t launch_scale_rhs(const Dims& d, const Dims& du, double factor, const double* rho, int dt,
                             void* fs, cudaStream_t s);

// phi64 += e * inv_scale on interior nodes
cudaError_t launch_correct(const Dims& d, int dt_e, const void* e, double inv_scale, double* phi,
                           const DevState* st, cudaStream_t s);

// out = A phi (unscaled) on interior nodes, storage dt
cudaError_t launch_apply(const Dims& d, int order, const double h[3], int dt, const void* phi,
                         void* out, cudaStream_t s);

// Single-CTA CG on the coarsest level: solves -A e = d * fs (zero boundary).
cudaError_t launch_coarse_cg(const Dims& d, int order, const double h[3], int dt_fs,
                             const void* fs, int dt_e, void* e, double tol, int max_iter,
                             DevState* st, cudaStream_t s);
size_t coarse_cg_smem_bytes(const Dims& d);

// Sum the per-block partials of a delta pass into the state and decide
// convergence.  mode: 0 = record reference norm, 1 = record initial residual,
// 2 = iteration check (iter += 1), 3 = IR outer check (also sets the scale).
// cond/chunk: when chunk > 0 the kernel runs inside a CUDA-graph while loop and
// sets its condition (continue while not done and iter % chunk != 0).
cudaError_t launch_finish_norm(const double* partials, int nblocks, double dscale, int mode,
                               DevState* st, cudaStream_t s, unsigned long long cond = 0,
                               int chunk = 0);

// ---------------------------------------------------------------- CG (FP64)
// r = d * delta(phi)  (SPD residual), p = r, partials of r.r
cudaError_t launch_cg_init(const Dims& d, int order, const double h[3], const double* phi,
                           const double* fs, double* r, double* p, double* partials,
                           LaunchCfg* cfg, cudaStream_t s);
// q = -A p, partials of p.q
cudaError_t launch_cg_apply(const Dims& d, int order, const double h[3], const double* p,
                            double* q, double* partials, const DevState* st, cudaStream_t s);
// x += alpha p; r -= alpha q; partials of r.r
cudaError_t launch_cg_update(const Dims& d, double* x, double* r, const double* p, const double* q,
                             double* partials, const DevState* st, cudaStream_t s);
// p = r + beta p
cudaError_t launch_cg_pupdate(const Dims& d, const double* r, double* p, const DevState* st,
                              cudaStream_t s);
// scalar steps: which = 0: alpha = rho/pq; 1: convergence + beta (CG); 2: start;
// 3: convergence only (PCG); 4: PCG beta = r.z/rho; 5: PCG start, rho = r.z
cudaError_t launch_cg_scalar(const double* partials, int nblocks, int which, DevState* st,
                             cudaStream_t s, unsigned long long cond = 0, int chunk = 0);
// PCG (Sec. 2.1.2): z = B^-1 r with the multicolour symmetric Gauss-Seidel
// preconditioner (pcg_precond_kernels(order) launches; skipped once st->done);
// the last pass writes per-block partials {r.z, 0} (pcg_partials_count blocks).
cudaError_t launch_pcg_precond(const Dims& d, int order, const double h[3], const double* r, double* z,
                               double* partials, const DevState* st, cudaStream_t s);
int pcg_partials_count(const Dims& d, int order);
int pcg_precond_kernels(int order);

int cart_partials_count(const Dims& d);

// st->chunk_end = st->iter + k: iteration budget of the next loop-graph launch
cudaError_t launch_set_budget(DevState* st, int k, cudaStream_t s);
// out[i] = x[i] * 2^e rounded to the nearest FP32 (ties to even), |e| <= 100
// phi[i] += e[i] * 2^p (|p| <= 100) on n elements: the refinement's correction.
cudaError_t launch_add_pow2_f32(const float* e, long long n, int p, double* phi, cudaStream_t s);
cudaError_t launch_pow2_to_f32(const double* x, long long n, int e, float* out, cudaStream_t s);
// reset a solve's state on the device (no host round trip)
cudaError_t launch_init_state(DevState* st, double tol, int max_iter, cudaStream_t s);
// first node of a loop graph: sets the while condition from the state
cudaError_t launch_loop_gate(const DevState* st, unsigned long long cond, cudaStream_t s);

}  // namespace ps
