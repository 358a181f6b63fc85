/*
 * poisson.h -- C ABI of the GB300 (sm_103a) library for matrix-free iterative
 * solution of the Poisson equation for the gravitational potential,
 *
 *     laplacian(Phi) = 4 pi G rho                      (Eq. 1 Cartesian, Eq. 2 spherical)
 *
 * after "Iterative Poisson Solvers for Self-gravity with the GPU Code Astaroth"
 * (arXiv 2605.03563).  Solvers: multicolour SOR / Gauss-Seidel (Sec. 2.1.1),
 * CG and Jacobi-preconditioned BiCGSTAB (Sec. 2.1.2), geometric multigrid
 * V-cycles (Sec. 2.1.3); open boundary by multipole expansion (Sec. 2.2,
 * Eqs. outer_expansion and outer_multipole).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers named *_dev are device pointers (cudaMalloc or torch tensors on the
 * current device); pointers named *_host are host pointers.  The caller owns
 * every buffer it passes; the library owns what a handle allocates and frees
 * it in poisson_destroy.  `stream` is a cudaStream_t; NULL is CUDA's default
 * stream, so work is ordered after what the caller enqueued there.
 *
 * Cartesian fields: contiguous, x fastest, extents (n[a] + 2g - 1) per axis,
 * where g = stencil_order / 2 is the stencil radius; node i of axis a (node 0
 * and node n[a] are the boundary, 1..n[a]-1 the unknowns) sits at array index
 * i + g - 1.  The non-interior layers of phi carry Dirichlet data (given, or
 * written by the multipole boundary).  "N^3" means N intervals per axis.
 *
 * Spherical fields: extents (Nr+2, Ntheta+2, Nphi+2) with r fastest; node
 * (i,j,k) sits at array index (i+1, j+1, k+1); array index 0 / Nr+1 along r
 * are the inner mirror ghost and the outer Dirichlet ghost.
 *
 * Errors: every call returns a ps_status; nothing is thrown and nothing
 * aborts.  poisson_last_error() returns a thread-local message describing the
 * last failure.  Argument errors are detected before any GPU work.
 */
#ifndef POISSON_GB300_H
#define POISSON_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PS_OK = 0,
  PS_ERR_INVALID_ARG = 1,   /* bad shape, order, method, l_max, pointer ... */
  PS_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement */
  PS_ERR_OOM = 3,           /* device allocation failed */
  PS_ERR_CUDA = 4,          /* a CUDA runtime call failed (message has the text) */
  PS_NOT_CONVERGED = 5,     /* max_iter reached; phi and info are valid (Sec. 2.1) */
  PS_DIVERGED = 6,          /* residual became NaN/Inf or grew 1e3-fold */
  PS_ERR_TIMEOUT = 7        /* a bounded device wait ran out */
} ps_status;

typedef enum { PS_GRID_CART_UNIFORM = 0, PS_GRID_SPHERICAL = 1 } ps_grid_kind;

/* Cartesian: n = intervals per axis, lo/hi = box corners (uniform spacing
 * h[a] = (hi[a]-lo[a])/n[a]).  Spherical: n = node counts (Nr, Ntheta, Nphi);
 * lo/hi are ignored (the coordinates come from poisson_create's coords). */
typedef struct {
  int32_t kind;
  int32_t n[3];
  double lo[3];
  double hi[3];
} ps_grid;

typedef enum { PS_BC_DIRICHLET_GIVEN = 0, PS_BC_MULTIPOLE = 1 } ps_outer_bc;
/* Inner radial boundary of a spherical grid (Cartesian grids take PS_INNER_NONE):
 * PS_INNER_NEUMANN: mirror ghost Phi_{-1} = Phi_1 at r_{-1} = 2 r_0 - r_1;
 * PS_INNER_MULTIPOLE: Dirichlet ghost at r_{-1} from the inner expansion
 *   Phi = -G sum qbar_lm r^l sqrt(4 pi/(2l+1)) Y_lm (Eq. inner_expansion) with
 *   qbar_lm = sum rho dV sqrt(4 pi/(2l+1)) Y_lm / r'^(l+1) (Eq. inner_multipole)
 *   over the unknown nodes (Sec. 2.2, for r_in > 0; zero-pad the density near
 *   r_in for accuracy).  Needs l_max >= 0 and r_{-1} > 0. */
typedef enum { PS_INNER_NONE = 0, PS_INNER_NEUMANN = 1, PS_INNER_MULTIPOLE = 2 } ps_inner_bc;

/* origin: expansion centre of the multipole boundary (Cartesian; Sec. 2.2
 * recommends keeping it near the centre of mass); the spherical grid always
 * expands about r = 0.  G: gravitational constant of Eq. 1. */
typedef struct {
  int32_t outer;
  int32_t inner;
  double origin[3];
  double G;
} ps_bc;

/* PS_SOR red-black / multicolour SOR (Sec. 2.1.1; Cartesian and spherical);
 * PS_CG conjugate gradients (Sec. 2.1.2); PS_PCG CG preconditioned by
 * multicolour Gauss-Seidel (Sec. 2.1.2) in its symmetric form
 * B = (D + L) D^-1 (D + U), D, L, U the blocks of -A in colour order, applied
 * as colour passes ascending then descending (2, 3 colours for the 7-, 13-point
 * stencils); PS_MG geometric multigrid (Sec. 2.1.3); PS_BICGSTAB right-Jacobi
 * BiCGSTAB (spherical grids).  CG and PCG stop on the unpreconditioned
 * residual and run in FP64. */
typedef enum { PS_SOR = 0, PS_CG = 1, PS_MG = 2, PS_BICGSTAB = 3, PS_PCG = 4 } ps_method;

/* PS_FP64: every kernel computes and stores in FP64.
 * PS_MIXED_FP32: Cartesian: FP64 iterative refinement (outer residual,
 *   correction, norms, multipole moments and coarsest solve in FP64) around
 *   FP32 inner V-cycles.  Spherical: FP64 iterative refinement around inner
 *   BiCGSTAB solves with FP32 Krylov vectors (iterate, right-hand side, true
 *   residuals and dot products in FP64).  Each inner solve applies right-Jacobi
 *   BiCGSTAB to the volume-scaled correction equation V L e = V r (V the cell
 *   volume r^2 dr sin(theta), which makes the flux form symmetric and keeps the
 *   recursion free of the excursions that the unscaled one shows on graded
 *   grids), starts from the FP64 true residual r and runs until its recursive
 *   residual has dropped 2^-k-fold, k = inner_cycles (0 = 2); an inner solve
 *   whose FP32 recursion overflows is discarded and retried with half the
 *   iterations.  Convergence is decided on the FP64 true residual.
 * PS_MIXED_BF16: as PS_MIXED_FP32, with the finest inner level stored in BF16
 *   (Cartesian; spherical treats it as PS_MIXED_FP32).
 * Spherical BiCGSTAB in either precision stops on the true residual b - A x,
 * which replaces the recursively updated one at every hundredfold drop
 * (residual replacement). */
typedef enum { PS_FP64 = 0, PS_MIXED_FP32 = 1, PS_MIXED_BF16 = 2 } ps_precision;

typedef struct {
  int32_t method;        /* ps_method */
  int32_t prec;          /* ps_precision */
  double omega;          /* SOR weight (Sec. 2.1.1); MG smoothing uses 1 */
  int32_t nu1, nu2;      /* V(nu1,nu2) pre-/post-smoothing sweeps */
  int32_t max_iter;      /* SOR steps / CG or BiCGSTAB iterations / V-cycles / IR steps */
  int32_t inner_cycles;  /* Cartesian mixed modes: inner V-cycles per IR step; spherical
                            PS_MIXED_FP32: the inner solve's reduction 2^-inner_cycles (0 = 2) */
  void* stream;          /* cudaStream_t; NULL = CUDA's default stream */
  int32_t tile_min_n;    /* Cartesian MG, mixed modes: FP32/BF16 inner levels (other than the
                            coarsest) with at least this many intervals on every axis run the
                            TMA-staged tile kernels (fused two-colour sweep for the 7-point
                            operator, fused residual + restriction); 0 = library default (16),
                            < 0 = never.  Results are bitwise the same either way.  FP64 levels
                            always use the per-colour passes. */
  int32_t sor_schedule;  /* PS_SOR weights (ps_sor_schedule): the given omega, the Chebyshev
                            sequence of Eq. omega_n, or omega_opt of Eq. 3; 0 = given omega */
  int32_t compact_order; /* PS_MG on a stencil_order 2 handle with equal spacings: 0 = the
                            7-point stencil with red-black Gauss-Seidel (above); 2, 4 or 6 =
                            the compact radius-one discretisation of that order (Sec. 2.1.3),
                            L_h phi = R_h (4 pi G rho), smoothed by the SPAI smoother of
                            Eq. richardson with Table 1's coefficients, Galerkin coarse
                            operators R A P, coarsest level by CG; PS_FP64, or
                            PS_MIXED_FP32: FP64 refinement around FP32 inner V-cycles
                            (inner_cycles per step).  The relative residual is
                            ||R_h f - L_h phi|| / ||R_h f - L_h phi0||. */
  int32_t use_tuning;    /* Cartesian PS_MG: 1 = take nu1, nu2, inner_cycles, tile_min_n and the
                            fused sweep's tile shape from the handle's tuning for this precision
                            (poisson_set_tuning), when one is set; 0 = use the fields above */
} ps_solve_opts;

/* SOR weights (Sec. 2.1.1).  rJ is the Jacobi spectral radius estimate: Eq. 4
 * on Cartesian grids (interval counts and spacings of the grid), the local
 * Eq. local_rjac on spherical grids (unknown-node counts per axis, the radial
 * width (r_{i+1} - r_{i-1})/2 of the flux form, r_i dtheta, r_i sin(theta_j)
 * dphi), which makes the weights position-dependent there.
 *   PS_SOR_FIXED      ps_solve_opts.omega everywhere;
 *   PS_SOR_CHEBYSHEV  omega_1 = 1/(1 - rJ^2/2), omega_{n+1} = 1/(1 - rJ^2 omega_n/4)
 *                     (Eq. omega_n from n = 1), n advancing once per colour pass;
 *   PS_SOR_OPTIMAL    omega_opt = 2/(1 + sqrt(1 - rJ^2)) (Eq. 3).
 * ps_solve_opts.omega is ignored by the last two. */
typedef enum { PS_SOR_FIXED = 0, PS_SOR_CHEBYSHEV = 1, PS_SOR_OPTIMAL = 2 } ps_sor_schedule;

typedef struct {
  int32_t iterations;        /* steps taken (V-cycles, Krylov iterations, SOR steps, IR steps) */
  int32_t status;            /* ps_status of the solve */
  double rel_residual;       /* ||f - A phi||_2 / ||f - A phi0||_2, phi0 = boundary data only */
  double rho_conv;           /* Eq. rho: (||r_m|| / ||r_0||)^(1/m) */
  double t_mp_ms;            /* multipole boundary time (moments + faces) */
  double t_iter_ms;          /* iteration time */
  int64_t inner_cycles;      /* Cartesian mixed: total inner V-cycles; spherical mixed: residual replacements */
  int64_t coarse_iterations; /* MG: total CG iterations on the coarsest level */
  int64_t kernel_launches;   /* CUDA kernels this solve launched */
  double moments[81];        /* first min((l_max+1)^2, 81) multipole moments q_lm, index l*l+l+m */
} ps_info;

typedef struct ps_ctx* ps_handle;

/* ------------------------------------------------------------------ solves */

/* Build a solver for one grid.  Validates everything, builds the multigrid
 * level list (halving while every axis has an even interval count >= 16,
 * Sec. 2.1.3), allocates the device hierarchy and workspace, uploads the
 * 1-D coordinate tables and the multipole coefficient tables.
 *   grid           Cartesian or spherical description (see ps_grid)
 *   coords_host    NULL for Cartesian; spherical: three host arrays r[Nr],
 *                  theta[Ntheta], phi[Nphi] of node coordinates (r increasing,
 *                  theta_j = (j+1/2) pi / Ntheta, phi_k = 2 pi k / Nphi)
 *   stencil_order  2 (7-point) or 4 (13-point, Cartesian only)
 *   bc             boundary description (NULL = Dirichlet data given, G = 1)
 *   l_max          multipole order, 0..16 (ignored for given Dirichlet data)
 *   out            receives the handle
 * Returns PS_ERR_INVALID_ARG before allocating if anything is inconsistent. */
ps_status poisson_create(const ps_grid* grid, const double* const coords_host[3],
                         int stencil_order, const ps_bc* bc, int l_max, ps_handle* out);

/* Solve laplacian(phi) = 4 pi G rho to ||f - A phi|| <= tol * ||f - A phi0||.
 *   rho_dev   density on the field layout (FP64, read only)
 *   phi_dev   FP64 field: in = initial guess (unknowns) + Dirichlet data
 *             (boundary/ghost layers), out = solution (and, with the
 *             multipole boundary, the boundary values it used)
 *   opts      method, precision, smoothing, limits and stream (NULL = MG,
 *             FP64, V(2,2), max_iter 100)
 *   info      filled after an internal stream synchronisation (may be NULL)
 * Runs asynchronously on the stream except for the final synchronisation.
 * Returns PS_NOT_CONVERGED / PS_DIVERGED with phi holding the last iterate. */
ps_status poisson_solve(ps_handle h, const double* rho_dev, double* phi_dev, double tol,
                        const ps_solve_opts* opts, ps_info* info);

/* Asynchronous, steppable form of poisson_solve (continuous batching).  The
 * solve's state stays on the device between calls; its work runs on the
 * handle's own stream, ordered after what opts->stream held at begin, and
 * opts->stream waits for the copy-back enqueued by end.  One solve in flight
 * per handle; phi_dev and rho_dev must stay valid until end.
 *   begin  validates, enqueues the multipole boundary, right-hand side,
 *          reference and initial residual (no host synchronisation)
 *   step   enqueues up to max_iterations more iterations (one CUDA-graph
 *          launch whose device-side while loop stops at convergence)
 *   poll   waits for the handle's stream and reports *done (converged, not
 *          converged or diverged); info (may be NULL) gets the progress
 *   end    copies the iterate to phi_dev, waits, fills info and returns the
 *          solve's status exactly as poisson_solve does.
 * poisson_solve = begin, poll, (step, poll)*, end. */
ps_status poisson_solve_begin(ps_handle h, const double* rho_dev, double* phi_dev, double tol,
                              const ps_solve_opts* opts);
ps_status poisson_solve_step(ps_handle h, int max_iterations);
ps_status poisson_solve_poll(ps_handle h, int* done, ps_info* info);
ps_status poisson_solve_end(ps_handle h, ps_info* info);

/* Solve n independent requests, each with its own handle, density, potential
 * and tolerance.  Each request runs on its handle's stream, so the kernels of
 * different requests overlap on the GPU.  Results equal n separate
 * poisson_solve calls bit for bit; infos[i] receives request i's info.
 * Handles must be distinct. */
ps_status poisson_solve_batch(ps_handle* hs, const double* const* rho_dev, double* const* phi_dev,
                              const double* tol, int n, const ps_solve_opts* opts,
                              ps_info* infos);

/* Release the handle and everything it allocated (NULL is a no-op). */
void poisson_destroy(ps_handle h);

/* Tuned settings of a handle (no paper counterpart: the autotuner's output).
 * For one precision of Cartesian multigrid solves they replace the solve
 * options nu1, nu2 (V(nu1, nu2), Sec. 2.1.3), inner_cycles (inner V-cycles
 * per refinement step), tile_min_n and the tile shape of the TMA-staged fused
 * red-black sweep of FP32/BF16 levels whenever ps_solve_opts.use_tuning is 1:
 *   sweep_tile 0 = the storage type's default, 1 = 4 rows per warp x 4 warps
 *   (64 x 16 tile), 2 = 2 x 4 (64 x 8), 3 = 8 x 4 (64 x 32), 4 = 4 x 8 (64 x 32);
 * and the tile shape of the fused residual + restriction of FP32/BF16 7-point
 * levels:
 *   restrict_tile 0 = the default (3), 1 = 4 coarse rows per warp x 4 warps
 *   (32 x 16 coarse tile), 2 = 2 x 4 (32 x 8), 3 = 3 x 4 (32 x 12);
 * every shape gives the same result bit for bit.  The autotuner times whole
 * solves per (grid size, order, precision, tolerance) and a caller installs
 * its choice here; solves without use_tuning are unaffected. */
typedef struct {
  int32_t nu1, nu2;        /* >= 0, nu1 + nu2 >= 1 */
  int32_t inner_cycles;    /* >= 1 (mixed precisions) */
  int32_t tile_min_n;      /* as ps_solve_opts.tile_min_n */
  int32_t sweep_tile;      /* 0 .. 4 */
  int32_t restrict_tile;   /* 0 .. 3 */
} ps_tuning;

/* Install (t != NULL) or clear (t == NULL) the tuning of precision prec
 * (ps_precision) on handle h.  Host only; PS_ERR_INVALID_ARG for a NULL or
 * spherical handle, an unknown precision or out-of-range fields. */
ps_status poisson_set_tuning(ps_handle h, int prec, const ps_tuning* t);

/* *is_set = 1 and *out = the tuning of precision prec if one is installed,
 * else *is_set = 0 (out untouched).  Host only. */
ps_status poisson_get_tuning(ps_handle h, int prec, ps_tuning* out, int* is_set);

/* Thread-local text of the last error (never NULL; "" when none). */
const char* poisson_last_error(void);

/* Device bytes poisson_create + poisson_solve would allocate for this grid and
 * precision (used for admission control); 0 for invalid arguments. */
size_t poisson_workspace_bytes(const ps_grid* grid, int stencil_order, int l_max, int prec);

/* Operators of the compact-stencil multigrid (Sec. 2.1.3), computed on the
 * host exactly as a compact solve builds them (no GPU work).  For compact
 * order 2, 4 or 6 and finest spacing h > 0, level l = 0 .. nlevels-1 has
 * spacing h 2^l and
 *   a[4 l .. 4 l + 3]  the class weights (centre, faces, edges, corners;
 *                      absolute units) of its operator: the compact L_h on
 *                      level 0, the Galerkin product R A P of the level above
 *                      (full weighting R, trilinear P = 8 R^T) below it;
 *   m[4 l .. 4 l + 3]  the SPAI smoother M = h_l^2 (alpha, beta, gamma, delta)
 *                      of Table 1 (Eq. Smoother);
 *   omega[l]           its relaxation weight (Eq. richardson).
 * All three are host arrays owned by the caller; m and omega may be NULL.
 * Errors: PS_ERR_INVALID_ARG for an order other than 2, 4, 6, h <= 0 or not
 * finite, nlevels < 1 or > 30, or a NULL a. */
ps_status poisson_compact_operators(int order, double h, int nlevels, double* a, double* m, double* omega);

/* ------------------------------------------------------------------ batched executor
 * Many Cartesian multigrid solves of different grid sizes advanced together
 * (continuous batching): one step advances every active solve by the same
 * number of V-cycles (FP64) or refinement steps (PS_MIXED_FP32) through one
 * launch of a captured CUDA graph whose phase kernels (colour passes, residual,
 * full weighting, coarsest CG, prolongation, norm) walk device-resident work
 * lists of (solve, level, tile) items.  Adding or removing a solve only rewrites
 * those lists; the graph, captured once per iteration count, serves any mix of
 * sizes.  Each solve runs the V(nu1, nu2) iteration of Sec. 2.1.3 on its own
 * handle's hierarchy, with its own reductions: its result does not depend on
 * what else is in the batch, and equals a separate poisson_solve up to the
 * rounding of the norms and of the coarsest CG's dot products (different
 * reduction trees).  Sweeps always use the per-colour passes.
 * Calls on one batch must not overlap; a handle added to a batch must not be
 * used for anything else until it is removed. */
typedef struct ps_batch_ctx* ps_batch;

/* capacity: slots (1..1024); max_n: largest interval count per axis of the
 * grids that will be added (16..8192; sets the number of level phases);
 * stencil_order 2 or 4; prec PS_FP64 or PS_MIXED_FP32 (FP64 refinement around
 * FP32 inner V-cycles, inner_cycles per step); nu1 >= 1, nu2 >= 0. */
ps_status poisson_batch_create(int capacity, int max_n, int stencil_order, int prec, int nu1, int nu2,
                               int inner_cycles, ps_batch* out);
void poisson_batch_destroy(ps_batch b);

/* Start a solve in a free slot on handle h (Cartesian, same stencil order,
 * multigrid-able, coarsest level of at most 4096 unknowns): multipole boundary
 * or given boundary data, scaled right-hand side and initial residual are
 * enqueued after the caller's work on CUDA's default stream.  rho_dev / phi_dev
 * as for poisson_solve; they must stay valid until poisson_batch_remove.
 * *slot receives the slot index.  PS_ERR_INVALID_ARG when the batch is full. */
ps_status poisson_batch_add(ps_batch b, ps_handle h, const double* rho_dev, double* phi_dev, double tol,
                            int max_iter, int* slot);

/* Enqueue `iterations` (1..64) iterations of every active solve (one graph
 * launch; no host synchronisation).  Finished solves are skipped. */
ps_status poisson_batch_step(ps_batch b, int iterations);

/* Wait for the batch and report every slot: status[i] = -1 free, 0 running,
 * 1 converged, 2 iteration budget exhausted, 3 diverged, 4 fault;
 * iterations[i] (optional) = iterations taken.  Arrays hold `capacity` entries. */
ps_status poisson_batch_poll(ps_batch b, int32_t* status, int32_t* iterations);

/* End the solve in `slot`: copies the potential to the caller's phi (ordered
 * before later work on CUDA's default stream), fills info (may be NULL) and
 * frees the slot.  Returns PS_OK, PS_NOT_CONVERGED or PS_DIVERGED like
 * poisson_solve. */
ps_status poisson_batch_remove(ps_batch b, int slot, ps_info* info);

/* ------------------------------------------------------------------ kernel timing
 * Opt-in timing of the hot kernels of a handle's solves with CUDA events
 * recorded on the solve stream around each launch (finest-level sweeps,
 * residual/restriction/prolongation passes, convergence norms, coarsest
 * solve, multipole moments and boundary values).  Each record carries the
 * algorithmic bytes (minimal HBM traffic of the operation) and FP64/FP32
 * arithmetic operations of one launch.  No paper counterpart: measurement
 * support for the roofline figures. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
  double bytes_per_launch;   /* algorithmic bytes of one launch (mean over the class's launches) */
  double ops_per_launch;     /* arithmetic instructions of one launch (FMA = 1; mean) */
  int32_t fp64;              /* 1 when the arithmetic runs on the FP64 pipe */
  int32_t variant;           /* tile shape of the last timed launch (fused sweeps: 1..4), else 0 */
} ps_kernel_stat;

/* enable != 0 starts recording (events are created lazily; at most 16384
 * launches are recorded between reads); 0 stops. */
ps_status poisson_profile_enable(ps_handle h, int enable);

/* Synchronises the handle's stream, folds the recorded launches into per-kernel
 * totals, writes up to max entries and returns how many kernels were seen
 * (negative on error).  Recorded launches are cleared. */
int poisson_profile_read(ps_handle h, ps_kernel_stat* out, int max);

/* ------------------------------------------------------------------ op-level calls
 * Single kernels of the hot path on caller-owned buffers, for validation and
 * benchmarking.  dtype: 0 = FP64, 1 = FP32, 2 = BF16 storage (arithmetic in
 * FP64 for FP64 storage, FP32 otherwise).  Cartesian fields follow the layout
 * above.  Each call is asynchronous on `stream` unless it returns a host value. */

/* out = A phi on interior nodes (7-point or 13-point Laplacian, Eq. 1 with
 * the stencils of Sec. 2.1); non-interior entries of out are left untouched. */
ps_status ps_op_apply(const ps_grid* grid, int stencil_order, int dtype, const void* phi_dev,
                      void* out_dev, void* stream);

/* r = f - A phi on interior nodes and ||r||_2^2 (FP64, deterministic) into
 * *norm2_host (synchronises; pass NULL to skip). */
ps_status ps_op_residual(const ps_grid* grid, int stencil_order, int dtype, const void* phi_dev,
                         const void* f_dev, void* r_dev, double* norm2_host, void* stream);

/* Allocation-free variant of ps_op_residual for FP64 fields (the paper has no
 * counterpart; this is an integration aid).  For callers that must not
 * allocate device memory -- code whose device memory is owned by an external
 * pool or arena, latency-critical loops where an allocation may stall or
 * fail, hosts with a no-allocation policy.  It computes the same r = f - A phi
 * on interior nodes and ||r||_2^2 but calls no cudaMalloc/cudaFree: its scratch
 * (per-block partial sums) is one fixed 256 KB array in device global memory
 * that every device loading the library keeps until exit.  When norm2_host is
 * non-NULL, ||r||^2 is copied back and the stream is synchronised; with NULL
 * the call is asynchronous and ||r||^2 stays only in the shared scratch.
 *   - Grids whose launch needs more than 32768 thread blocks (beyond about
 *     512^3 intervals) are rejected with PS_ERR_INVALID_ARG before GPU work.
 *   - All calls on a device share that array: calls whose kernels can
 *     overlap on the GPU race on it and must be serialised by the caller.
 *   - The first call on each device looks up the array's device address with
 *     that device current; make it before any stream capture.  The address is
 *     kept for the life of the process: after cudaDeviceReset (or any other
 *     teardown of the device's primary context) it is stale, so do not call
 *     this entry point on that device again in the same process. */
ps_status ps_op_residual_noalloc(const ps_grid* grid, int stencil_order, const double* phi_dev,
                                 const double* f_dev, double* r_dev, double* norm2_host,
                                 void* stream);

/* One multicolour SOR step in place (Sec. 2.1.1): colours (i+j+k) mod 2 for
 * order 2, mod 3 for order 4, ascending; phi += omega (phi_GS - phi). */
ps_status ps_op_sweep(const ps_grid* grid, int stencil_order, int dtype, void* phi_dev,
                      const void* f_dev, double omega, void* stream);

/* Full-weighting restriction (Sec. 2.1.3) of the interior of r_fine_dev onto
 * the interior of f_coarse_dev (grid = the fine grid; coarse = n/2). */
ps_status ps_op_restrict(const ps_grid* fine_grid, int stencil_order, int dtype,
                         const void* r_fine_dev, void* f_coarse_dev, void* stream);

/* The same full weighting for a 7-point residual that is exactly zero on the
 * black nodes ((i+j+k) odd, node indices), as a complete red-black
 * Gauss-Seidel sweep leaves it (Sec. 2.1.1, 2.1.3): the zero terms are not
 * summed.  On such input the result equals ps_op_restrict's bit for bit, up
 * to the sign of zero values; on other input it is not a restriction.
 * stencil_order must be 2; dtype FP64 or FP32. */
ps_status ps_op_restrict_red(const ps_grid* fine_grid, int stencil_order, int dtype,
                             const void* r_fine_dev, void* f_coarse_dev, void* stream);

/* phi_fine += P e_coarse with P = 8 R^T (trilinear, Sec. 2.1.3); coarse
 * boundary values are treated as zero (grid = the fine grid). */
ps_status ps_op_prolong(const ps_grid* fine_grid, int stencil_order, int dtype,
                        const void* e_coarse_dev, void* phi_fine_dev, void* stream);

/* out[i] = x[i] * 2^e rounded to the nearest FP32 value (ties to even), for
 * finite x and -100 <= e <= 100 (otherwise PS_ERR_INVALID_ARG).  This is the
 * conversion the mixed-precision multigrid (Sec. 2.1.3) applies when it stores
 * the scaled FP64 residual as the FP32/BF16 inner right-hand side; it runs on
 * the integer pipe.  x_dev and out_dev are device arrays of n elements owned by
 * the caller. */
ps_status ps_op_scale_to_fp32(const double* x_dev, int64_t n, int e, float* out_dev, void* stream);

/* phi[i] += e[i] * 2^p for -100 <= p <= 100 (otherwise PS_ERR_INVALID_ARG): the
 * correction step of the mixed-precision refinement (Sec. 2.1.3), which adds
 * the FP32 inner solution, computed for a right-hand side scaled by 2^-p, to
 * the FP64 potential.  e * 2^p is exact in FP64 and is built on the integer
 * pipe; the sum rounds once, as fma((double)e, 2^p, phi) does.  e_dev (FP32)
 * and phi_dev (FP64) are device arrays of n elements owned by the caller. */
ps_status ps_op_add_scaled_fp32(const float* e_dev, int64_t n, int p, double* phi_dev, void* stream);

/* Multipole moments q_lm (Eq. outer_multipole) of rho over the interior nodes
 * about `origin`, (l_max+1)^2 doubles into q_host (synchronises). */
ps_status ps_op_multipole_moments(const ps_grid* grid, int stencil_order, const double* rho_dev,
                                  const double origin[3], int l_max, double* q_host,
                                  void* stream);

/* Eq. outer_expansion written on every non-interior node of phi_dev. */
ps_status ps_op_multipole_boundary(const ps_grid* grid, int stencil_order, const double* q_host,
                                   const double origin[3], int l_max, double G, double* phi_dev,
                                   void* stream);

/* Spherical operator (Eq. 2 in flux form) applied to phi_dev (ghosted layout):
 * out = L phi on every unknown node, using phi's outer ghost as given, the
 * inner mirror ghost and periodic phi (ghost slots of phi are read, not
 * written).  Uses the coordinates of handle h (spherical). */
ps_status ps_op_spherical_apply(ps_handle h, const double* phi_dev, double* out_dev, void* stream);

/* ------------------------------------------------------------------ measurement support
 * FP64 pipe throughput probe (no paper counterpart: it supplies the measured
 * peak against which the FP64-bound kernels' rooflines are stated).  Launches
 * `blocks` blocks of 256 threads; each thread runs 8 independent chains of
 * `iters` FP64 instructions -- fused multiply-adds for kind 0, adds for kind 1
 * -- and each block writes one double to out_dev[block] (device array of
 * `blocks` doubles owned by the caller).  *instructions_host (may be NULL)
 * receives the number of FP64 instructions the launch issues (warp lanes
 * counted one by one); the caller times the launch on `stream`.
 * Errors: PS_ERR_INVALID_ARG for kind not 0/1, blocks outside 1..2^20, iters
 * outside 1..2^24 or a NULL out_dev; PS_ERR_CUDA if the launch fails. */
ps_status ps_probe_fp64(int kind, int blocks, int iters, double* out_dev, double* instructions_host,
                        void* stream);

/* Failure-detection check of the bounded device waits (no paper counterpart).
 * The TMA tile kernels wait on mbarriers with a time limit read from the
 * global timer: 2 s for a kernel's first failing wait, 1 ms for every wait
 * after one has failed; a wait that runs out marks the kernel faulty and the
 * solve ends with PS_ERR_TIMEOUT instead of hanging the GPU.  This call runs
 * exactly that wait in one warp on an mbarrier that nothing ever arrives at
 * (first_wait != 0: the 2 s limit; 0: the 1 ms limit), synchronises `stream`
 * and returns PS_ERR_TIMEOUT with *waited_ms_host (may be NULL) = the time the
 * wait took.  out_dev: caller-owned device scratch of 3 int64.  No copy is in
 * flight and the context stays usable afterwards.  Errors: PS_ERR_INVALID_ARG
 * for a NULL out_dev, PS_ERR_CUDA if the launch or copy fails. */
ps_status ps_probe_bounded_wait(int first_wait, long long* out_dev, double* waited_ms_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* POISSON_GB300_H */
