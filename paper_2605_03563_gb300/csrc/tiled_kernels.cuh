// Host launchers of the TMA-staged z-marching tile kernels (tiled_kernels.cu).
// They need library-layout level arrays (rows padded so that every row starts
// on a 16-byte boundary, base 16-byte aligned).
#pragma once
#include "cart_kernels.cuh"

namespace ps {

// One full red-black Gauss-Seidel sweep (omega = 1) of the 7-point operator
// (Sec. 2.1.1: red nodes, then black nodes) written out of place:
// phi_out = sweep(phi_in).  Bitwise equal to the two in-place colour passes of
// launch_sweep_colour.  phi_out must hold the same boundary values as phi_in.
// Returns cudaErrorNotSupported for the 13-point operator.  Skipped entirely
// once st->done (if st is given).  fault (optional): set to 1 if a tile copy
// did not arrive in time.  tile: 0 (the storage type's default) or one of the
// kRbSweepTiles compiled tile shapes (see rb_sweep_default_tile); every shape
// gives the same result bit for bit.
constexpr int kRbSweepTiles = 4;
int rb_sweep_default_tile(int dt);
cudaError_t launch_rb_sweep(const Dims& d, int order, const double h[3], int dt, const void* phi_in,
                            void* phi_out, const void* fs, const DevState* st, int* fault,
                            cudaStream_t s, int tile = 0);

// Fused residual and full-weighting restriction (Sec. 2.1.3):
// fs_coarse = factor * R(phi_GS(phi) - phi) without storing the fine residual.
// Equal bit for bit to launch_delta into a buffer of the level's arithmetic
// type followed by launch_restrict.  tile: 0 (the storage type's default, see
// rr_default_tile) or one of the kRrTiles compiled tile shapes of the
// register-blocked FP32/BF16 7-point kernel (ignored by the 13-point and FP64
// kernel); every shape gives the same result bit for bit.
constexpr int kRrTiles = 3;
int rr_default_tile(int dt);
cudaError_t launch_resid_restrict(const Dims& fine, const Dims& coarse, int order, const double h[3], int dt_f,
                                  const void* phi, const void* fs, int dt_c, void* fs_c,
                                  double factor, int* fault, cudaStream_t s, int tile = 0);

// Residual norm pass after a completed omega = 1 colour sweep: nodes of the
// last colour have delta = 0 exactly (the residual kernel repeats the sweep's
// arithmetic on unchanged operands), so only the other colours are evaluated.
// Writes per-block partials {sum delta^2, 0}; returns the block count in nblocks.
cudaError_t launch_delta_colours(const Dims& d, int order, const double h[3], const double* phi,
                                 const double* fs, double* partials, int* nblocks, cudaStream_t s);
int delta_colours_partials(const Dims& d, int order);

}  // namespace ps
