// Batched multigrid executor: device-side descriptors, work lists and the
// launchers of its phase kernels (batch.cu).
//
// A batch holds up to `capacity` Cartesian multigrid solves of different grid
// sizes (each on its own handle's hierarchy).  One step advances every active
// solve by the same number of V-cycles (FP64) or refinement steps (mixed
// FP32): a fixed sequence of phase launches -- colour passes, residual,
// restriction, coarsest CG, prolongation, norm -- per level index, captured once
// into a plain CUDA graph.  Each phase kernel walks a device-resident work list
// with a grid-stride loop over the list's tiles; an entry of the list holds one
// solve's tiles of one level, and a block finds the entry of its tile by binary
// search over the prefix offsets.  So the same graph serves any mix of grid
// sizes, and a change of the batch's composition only rewrites small lists and
// the slot descriptors.  Tiles of finished solves are skipped.
#pragma once
#include "cart_kernels.cuh"

namespace ps {

static constexpr int PS_BMAX_LEVELS = 12;

// One level of one solve.
struct BLevel {
  Dims d;
  Coef<double> cf64;   // FP64 levels (and the coarsest CG)
  Coef<float> cf32;    // FP32 levels
  void* phi;
  void* fs;
  void* tmp;           // residual fed to the restriction
  int dt;              // storage of phi and fs (DT_F64 or DT_F32)
  int iso;             // equal spacing on all axes
  int zc;              // planes per tile along z
  int pad_;
};

// One solve.
struct BSlot {
  BLevel lv[PS_BMAX_LEVELS];
  DevState* st;
  double* partials;    // per-tile {sum, max} of this solve's norm pass
  double* phi64;       // finest FP64 potential (library layout)
  double* fs64;        // finest FP64 scaled right-hand side
  Coef<double> cf0;    // finest-level FP64 coefficients
  double dscale;       // d of the finest level (r = -d delta)
  int nlev;
  int nparts;          // partials written by the norm pass
  int active;
  int pad_;
};

// One solve's share of a list: `tiles` tiles of level `level` (a gx x gy x gz
// grid of tiles, x fastest), numbered first .. first+tiles-1 within the list.
// A tile's number inside its solve is also the index of its norm partial.
struct BItem {
  int slot, level, first, tiles, gx, gy;
};

// off/count: entries of the list; total: tiles over all entries.
struct BList {
  int off, count, total, pad_;
};

// Work-list kinds; list index = kind * PS_BMAX_LEVELS + level.
enum BListKind {
  BL_SWEEP = 0,   // colour-pass tiles of level l (also the residual before restriction)
  BL_COARSE_PT,   // point tiles of level l+1 (restriction target, zeroing)
  BL_CELLS,       // coarse cells of level l+1 (prolongation into level l)
  BL_CG,          // one item per solve whose coarsest level is l
  BL_NORM0,       // level-0 tiles of the norm after a sweep (FP64 batches), level index 0
  BL_PT0,         // level-0 point tiles (refinement: zero, correct, outer residual), level index 0
  BL_SLOTS,       // one item per active solve, level index 0
  BL_NKINDS
};

// Tile geometry (32 x 8 threads): number of tiles of each kind on a level.
void batch_tiles_sweep(const Dims& d, int order, int zc, int* gx, int* gy, int* gz);
void batch_tiles_points(const Dims& d, int zc, int* gx, int* gy, int* gz);
void batch_tiles_cells(const Dims& coarse, int zc, int* gx, int* gy, int* gz);
int batch_zchunk(const Dims& d);
// norm partials a batch writes for a solve whose finest level is d (one per
// level-0 sweep or point tile, whichever is more)
int batch_norm_partials(const Dims& d, int order);

// Phase launches (grid-stride over list `list`).  Every launcher takes the
// descriptor and work-list arrays in device memory.
struct BArgs {
  const BSlot* slots;
  const BItem* items;
  const BList* lists;
};
cudaError_t launch_b_sweep(const BArgs& a, int order, int dt, int list, int colour, cudaStream_t s);
cudaError_t launch_b_delta_skip(const BArgs& a, int order, int dt, int list, cudaStream_t s);
cudaError_t launch_b_restrict(const BArgs& a, int dt, int list, cudaStream_t s);
cudaError_t launch_b_prolong(const BArgs& a, int dt, int list, cudaStream_t s);
cudaError_t launch_b_coarse(const BArgs& a, int order, int dt, int list, int max_blocks,
                            size_t smem, double tol, cudaStream_t s);
cudaError_t launch_b_norm(const BArgs& a, int order, int list, cudaStream_t s);
cudaError_t launch_b_finish(const BArgs& a, int list, int max_blocks, cudaStream_t s);
cudaError_t launch_b_zero(const BArgs& a, int dt, int list, cudaStream_t s);
cudaError_t launch_b_correct(const BArgs& a, int list, cudaStream_t s);
cudaError_t launch_b_delta_ir(const BArgs& a, int order, int list, cudaStream_t s);
// out[i] = {done, iter} of every slot (inactive slots: {-1, 0})
cudaError_t launch_b_gather(const BSlot* slots, int capacity, int* out, cudaStream_t s);
// kernels the step graph launches per iteration (for launch accounting)
int batch_kernels_per_iteration(int nlev_max, int order, int prec, int nu1, int nu2, int inner);

}  // namespace ps
