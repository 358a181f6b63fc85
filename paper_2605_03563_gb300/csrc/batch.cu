// Batched multigrid executor: phase kernels over work lists (see batch.cuh).
//
// Every kernel walks its list with a grid-stride loop over the list's tiles; a
// tile is 32 x 8 x zc nodes (or cells) of one level of one solve.  The per-node arithmetic is that of
// the per-solve kernels (colour pass, residual on the non-last colours, full
// weighting, trilinear prolongation, norm after a sweep, refinement residual),
// so a solve advanced in a batch follows the same iteration as alone.  Per-solve
// reductions go to the solve's own partials (one per tile, tile order fixed by
// the solve's geometry), so a solve's results do not depend on what else is in
// the batch.
#include <algorithm>

#include "batch.cuh"
#include "stencil.cuh"

namespace ps {

static constexpr int BBX = 32, BBY = 8;
// blocks of a tile phase launch (grid-stride): 8 per SM
static int bgrid() { return 8 * device_sm_count(); }

// planes per tile: deeper tiles on the larger levels cut the per-tile work-list
// lookups and edge loads (48 grids of 32^3..256^3 to 1e-10, FP32 refinement:
// 417 -> 439 solves/s against 8 planes from 64; FP64 247 -> 248)
int batch_zchunk(const Dims& d) {
  const int nk = d.nk();
  return nk >= 120 ? 32 : (nk >= 60 ? 16 : (nk >= 16 ? 4 : 1));
}

void batch_tiles_sweep(const Dims& d, int order, int zc, int* gx, int* gy, int* gz) {
  const int ncol = order == 2 ? 2 : 3;
  const int per_row = (d.ni() + ncol - 1) / ncol;
  *gx = (per_row + BBX - 1) / BBX;
  *gy = (d.nj() + BBY - 1) / BBY;
  *gz = (d.nk() + zc - 1) / zc;
}

void batch_tiles_points(const Dims& d, int zc, int* gx, int* gy, int* gz) {
  *gx = (d.ni() + BBX - 1) / BBX;
  *gy = (d.nj() + BBY - 1) / BBY;
  *gz = (d.nk() + zc - 1) / zc;
}

int batch_norm_partials(const Dims& d, int order) {
  const int zc = batch_zchunk(d);
  int sx, sy, sz, px, py, pz;
  batch_tiles_sweep(d, order, zc, &sx, &sy, &sz);
  batch_tiles_points(d, zc, &px, &py, &pz);
  return std::max(sx * sy * sz, px * py * pz);
}

void batch_tiles_cells(const Dims& coarse, int zc, int* gx, int* gy, int* gz) {
  *gx = (coarse.nx + BBX - 1) / BBX;
  *gy = (coarse.ny + BBY - 1) / BBY;
  *gz = (coarse.nz + zc - 1) / zc;
}

// The tile with list-wide number t: its entry, and (bx, by, bz, number in the solve).
struct BTile {
  int slot, level, bx, by, bz, local;
};
__device__ __forceinline__ BTile find_tile(const BItem* __restrict__ items, const BList& L, int t) {
  int lo = 0, hi = L.count - 1;
  while (lo < hi) {   // last entry with first <= t
    const int mid = (lo + hi + 1) >> 1;
    if (items[L.off + mid].first <= t) lo = mid;
    else hi = mid - 1;
  }
  const BItem e = items[L.off + lo];
  BTile r;
  r.slot = e.slot;
  r.level = e.level;
  r.local = t - e.first;
  r.bx = r.local % e.gx;
  const int q = r.local / e.gx;
  r.by = q % e.gy;
  r.bz = q / e.gy;
  return r;
}

template <typename C> __device__ __forceinline__ const Coef<C>& coef_of(const BLevel& lv);
template <> __device__ __forceinline__ const Coef<double>& coef_of<double>(const BLevel& lv) { return lv.cf64; }
template <> __device__ __forceinline__ const Coef<float>& coef_of<float>(const BLevel& lv) { return lv.cf32; }

template <int G, typename T, typename C>
__device__ __forceinline__ C gs_any(bool iso, const T* phi, long long p, long long sy, long long sz,
                                    const Coef<C>& cf, C fs) {
  return iso ? gs_value<G, true>(phi, p, sy, sz, cf, fs) : gs_value<G, false>(phi, p, sy, sz, cf, fs);
}

// ------------------------------------------------------------------ colour pass (omega = 1)
template <int G, typename T>
__global__ void __launch_bounds__(BBX* BBY) kb_sweep(BArgs a, int list, int colour) {
  using C = typename St<T>::C;
  using S = St<T>;
  constexpr int NCOL = G == 1 ? 2 : 3;
  const BList L = a.lists[list];
  for (int it = blockIdx.x; it < L.total; it += gridDim.x) {
    const BTile item = find_tile(a.items, L, it);
    const BSlot& sl = a.slots[item.slot];
    if (sl.st->done) continue;
    const BLevel& lv = sl.lv[item.level];
    const Dims d = lv.d;
    const Coef<C> cf = coef_of<C>(lv);
    T* phi = (T*)lv.phi;
    const T* fs = (const T*)lv.fs;
    const int t = item.bx * BBX + threadIdx.x;
    const int jn = item.by * BBY + threadIdx.y + 1;
    if (jn > d.nj()) continue;
    const int kn0 = item.bz * lv.zc + 1, kn1 = min(kn0 + lv.zc, d.nk() + 1);
    const long long sy = d.sy(), sz = d.sz();
    for (int kn = kn0; kn < kn1; kn++) {
      const int r0 = ((colour - jn - kn - 1) % NCOL + NCOL) % NCOL;
      const int in = 1 + r0 + NCOL * t;
      if (in > d.ni()) continue;
      const long long p = d.at(in + G - 1, jn + G - 1, kn + G - 1);
      S::st(phi + p, gs_any<G>(lv.iso, phi, p, sy, sz, cf, S::ld(fs + p)));
    }
  }
}

// ------------------------------------------------------------------ residual after a sweep
// delta on the non-last colours, exact zeros on the last one (see k_delta_skip)
template <int G, typename T>
__global__ void __launch_bounds__(BBX* BBY) kb_delta_skip(BArgs a, int list) {
  using C = typename St<T>::C;
  using S = St<T>;
  constexpr int NCOL = G == 1 ? 2 : 3;
  const BList L = a.lists[list];
  for (int it = blockIdx.x; it < L.total; it += gridDim.x) {
    const BTile item = find_tile(a.items, L, it);
    const BSlot& sl = a.slots[item.slot];
    if (sl.st->done) continue;
    const BLevel& lv = sl.lv[item.level];
    const Dims d = lv.d;
    const Coef<C> cf = coef_of<C>(lv);
    const T* phi = (const T*)lv.phi;
    const T* fs = (const T*)lv.fs;
    T* out = (T*)lv.tmp;
    const int t = item.bx * BBX + threadIdx.x;
    const int jn = item.by * BBY + threadIdx.y + 1;
    if (jn > d.nj()) continue;
    const int kn0 = item.bz * lv.zc + 1, kn1 = min(kn0 + lv.zc, d.nk() + 1);
    const long long sy = d.sy(), sz = d.sz();
    for (int kn = kn0; kn < kn1; kn++) {
#pragma unroll
      for (int colour = 0; colour < NCOL; colour++) {
        const int r0 = ((colour - jn - kn - 1) % NCOL + NCOL) % NCOL;
        const int in = 1 + r0 + NCOL * t;
        if (in > d.ni()) continue;
        const long long p = d.at(in + G - 1, jn + G - 1, kn + G - 1);
        if (colour == NCOL - 1) {
          S::st(out + p, (C)0);
        } else {
          const C dl = gs_any<G>(lv.iso, phi, p, sy, sz, cf, S::ld(fs + p)) - S::ld(phi + p);
          S::st(out + p, dl);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ restriction
// item.level = fine level l; tile of coarse points of level l+1:
// fs_{l+1} = 4 R(delta_l) (full weighting) and phi_{l+1} = 0 (initial coarse guess).
template <typename T>
__global__ void __launch_bounds__(BBX* BBY) kb_restrict(BArgs a, int list) {
  using C = typename St<T>::C;
  using S = St<T>;
  const BList L = a.lists[list];
  for (int it = blockIdx.x; it < L.total; it += gridDim.x) {
    const BTile item = find_tile(a.items, L, it);
    const BSlot& sl = a.slots[item.slot];
    if (sl.st->done) continue;
    const BLevel& lf = sl.lv[item.level];
    const BLevel& lc = sl.lv[item.level + 1];
    const Dims fd = lf.d, cd = lc.d;
    const T* df = (const T*)lf.tmp;
    T* fsc = (T*)lc.fs;
    T* phic = (T*)lc.phi;
    const int I = item.bx * BBX + threadIdx.x + 1;
    const int J = item.by * BBY + threadIdx.y + 1;
    if (I > cd.ni() || J > cd.nj()) continue;
    const int K0 = item.bz * lc.zc + 1, K1 = min(K0 + lc.zc, cd.nk() + 1);
    const int g = fd.g;
    const long long sy = fd.sy(), sz = fd.sz();
    const C sc = (C)(4.0 / 64.0);
    for (int K = K0; K < K1; K++) {
      const long long c = fd.at(2 * I + g - 1, 2 * J + g - 1, 2 * K + g - 1);
      C plane[3];
#pragma unroll
      for (int dz = -1; dz <= 1; dz++) {
        C rows[3];
#pragma unroll
        for (int dy = -1; dy <= 1; dy++) {
          const long long q = c + dz * sz + dy * sy;
          rows[dy + 1] = (S::ld(df + q - 1) + S::ld(df + q + 1)) + (C)2 * S::ld(df + q);
        }
        plane[dz + 1] = (rows[0] + rows[2]) + (C)2 * rows[1];
      }
      const C acc = (plane[0] + plane[2]) + (C)2 * plane[1];
      const long long pc = cd.at(I + g - 1, J + g - 1, K + g - 1);
      S::st(fsc + pc, acc * sc);
      S::st(phic + pc, (C)0);
    }
  }
}

// ------------------------------------------------------------------ prolongation
// item.level = fine level l; tile of coarse cells of level l+1 (as k_prolong)
template <typename T>
__global__ void __launch_bounds__(BBX* BBY) kb_prolong(BArgs a, int list) {
  using C = typename St<T>::C;
  using S = St<T>;
  const BList L = a.lists[list];
  for (int it = blockIdx.x; it < L.total; it += gridDim.x) {
    const BTile item = find_tile(a.items, L, it);
    const BSlot& sl = a.slots[item.slot];
    if (sl.st->done) continue;
    const BLevel& lf = sl.lv[item.level];
    const BLevel& lc = sl.lv[item.level + 1];
    const Dims fd = lf.d, cd = lc.d;
    const T* ec = (const T*)lc.phi;
    T* phif = (T*)lf.phi;
    const int I = item.bx * BBX + threadIdx.x;
    const int J = item.by * BBY + threadIdx.y;
    if (I >= cd.nx || J >= cd.ny) continue;
    const int K0 = item.bz * lc.zc, K1 = min(K0 + lc.zc, cd.nz);
    const int g = fd.g;
    const long long csy = cd.sy(), csz = cd.sz();
    const long long fsy = fd.sy(), fsz = fd.sz();
    const C half = (C)0.5;
    for (int K = K0; K < K1; K++) {
      const long long c0 = cd.at(I + g - 1, J + g - 1, K + g - 1);
      C cc[2][2][2];
#pragma unroll
      for (int z = 0; z < 2; z++)
#pragma unroll
        for (int y = 0; y < 2; y++) {
          cc[z][y][0] = S::ld(ec + c0 + z * csz + y * csy);
          cc[z][y][1] = S::ld(ec + c0 + z * csz + y * csy + 1);
        }
      C vx[2][2][2];
#pragma unroll
      for (int z = 0; z < 2; z++)
#pragma unroll
        for (int y = 0; y < 2; y++) {
          vx[z][y][0] = cc[z][y][0];
          vx[z][y][1] = half * (cc[z][y][0] + cc[z][y][1]);
        }
      C vy[2][2][2];
#pragma unroll
      for (int z = 0; z < 2; z++)
#pragma unroll
        for (int q = 0; q < 2; q++) {
          vy[z][0][q] = vx[z][0][q];
          vy[z][1][q] = half * (vx[z][0][q] + vx[z][1][q]);
        }
      const long long f0 = fd.at(2 * I + g - 1, 2 * J + g - 1, 2 * K + g - 1);
#pragma unroll
      for (int cz = 0; cz < 2; cz++) {
        if (cz == 0 && K == 0) continue;
#pragma unroll
        for (int b = 0; b < 2; b++) {
          if (b == 0 && J == 0) continue;
#pragma unroll
          for (int q = 0; q < 2; q++) {
            if (q == 0 && I == 0) continue;
            const C v = cz == 0 ? vy[0][b][q] : half * (vy[0][b][q] + vy[1][b][q]);
            const long long p = f0 + cz * fsz + b * fsy + q;
            S::st(phif + p, S::ld(phif + p) + v);
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------ coarsest CG
// One block per solve whose coarsest level is item.level (the block's own item).
template <int G, typename T>
__global__ void __launch_bounds__(256) kb_coarse(BArgs a, int list, double tol) {
  extern __shared__ double p[];
  const BList L = a.lists[list];
  if ((int)blockIdx.x >= L.count) return;
  const BItem item = a.items[L.off + blockIdx.x];   // one tile per entry
  const BSlot& sl = a.slots[item.slot];
  if (sl.st->done) return;
  const BLevel& lv = sl.lv[item.level];
  const int nunk = lv.d.ni() * lv.d.nj() * lv.d.nk();
  if (lv.iso)
    coarse_cg_block<G, true, T, T, 16, 256>(lv.d, lv.cf64, (const T*)lv.fs, (T*)lv.phi, tol, nunk, sl.st, p);
  else
    coarse_cg_block<G, false, T, T, 16, 256>(lv.d, lv.cf64, (const T*)lv.fs, (T*)lv.phi, tol, nunk, sl.st, p);
}

// ------------------------------------------------------------------ norm after the post-smoothing (FP64)
// Level-0 tiles in the colour-pass geometry: delta on the non-last colours
// (the last colour's is exactly zero); one partial per tile.
template <int G>
__global__ void __launch_bounds__(BBX* BBY) kb_norm(BArgs a, int list) {
  constexpr int NCOL = G == 1 ? 2 : 3;
  __shared__ double sh[8];
  const BList L = a.lists[list];
  const int tid = threadIdx.x + BBX * threadIdx.y;
  for (int it = blockIdx.x; it < L.total; it += gridDim.x) {
    const BTile item = find_tile(a.items, L, it);
    const BSlot& sl = a.slots[item.slot];
    if (sl.st->done) continue;   // uniform over the block
    const BLevel& lv = sl.lv[0];
    const Dims d = lv.d;
    const double* phi = (const double*)lv.phi;
    const double* fs = (const double*)lv.fs;
    const int t = item.bx * BBX + threadIdx.x;
    const int jn = item.by * BBY + threadIdx.y + 1;
    const int kn0 = item.bz * lv.zc + 1, kn1 = min(kn0 + lv.zc, d.nk() + 1);
    const long long sy = d.sy(), sz = d.sz();
    double s2 = 0.0;
    if (jn <= d.nj()) {
      for (int kn = kn0; kn < kn1; kn++) {
#pragma unroll
        for (int colour = 0; colour < NCOL - 1; colour++) {
          const int r0 = ((colour - jn - kn - 1) % NCOL + NCOL) % NCOL;
          const int in = 1 + r0 + NCOL * t;
          if (in > d.ni()) continue;
          const long long q = d.at(in + G - 1, jn + G - 1, kn + G - 1);
          const double dl = gs_any<G>(lv.iso, phi, q, sy, sz, lv.cf64, fs[q]) - phi[q];
          s2 = fma(dl, dl, s2);
        }
      }
    }
    s2 = warp_sum(s2);
    if ((tid & 31) == 0) sh[tid >> 5] = s2;
    __syncthreads();
    if (tid < 32) {
      double v = tid < 8 ? sh[tid] : 0.0;
      v = warp_sum(v);
      if (tid == 0) {
        sl.partials[2 * item.local] = v;
        sl.partials[2 * item.local + 1] = 0.0;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ norm finisher
// One block per active solve (its own item): convergence check (mode 2).
__global__ void __launch_bounds__(1024) kb_finish(BArgs a, int list) {
  const BList L = a.lists[list];
  if ((int)blockIdx.x >= L.count) return;
  const BSlot& sl = a.slots[a.items[L.off + blockIdx.x].slot];
  finish_norm_block(sl.partials, sl.nparts, sl.dscale, 2, sl.st, 0ull, 0);
}

// ------------------------------------------------------------------ refinement pieces (mixed batches)
// zero the level's potential on a point tile (inner initial guess e = 0)
template <typename T>
__global__ void __launch_bounds__(BBX* BBY) kb_zero(BArgs a, int list) {
  const BList L = a.lists[list];
  for (int it = blockIdx.x; it < L.total; it += gridDim.x) {
    const BTile item = find_tile(a.items, L, it);
    const BSlot& sl = a.slots[item.slot];
    if (sl.st->done) continue;
    const BLevel& lv = sl.lv[item.level];
    const Dims d = lv.d;
    const int g = d.g;
    const int i = item.bx * BBX + threadIdx.x + g;
    const int j = item.by * BBY + threadIdx.y + g;
    if (i >= g + d.ni() || j >= g + d.nj()) continue;
    const int k0 = item.bz * lv.zc + g, k1 = min(k0 + lv.zc, g + d.nk());
    T* phi = (T*)lv.phi;
    for (int k = k0; k < k1; k++) phi[d.at(i, j, k)] = (T)0;
  }
}

// phi64 += e / scale (as k_correct), level-0 point tiles
__global__ void __launch_bounds__(BBX* BBY) kb_correct(BArgs a, int list) {
  const BList L = a.lists[list];
  for (int it = blockIdx.x; it < L.total; it += gridDim.x) {
    const BTile item = find_tile(a.items, L, it);
    const BSlot& sl = a.slots[item.slot];
    if (sl.st->done) continue;
    const BLevel& lv = sl.lv[0];
    const Dims d = lv.d;
    const double isc = inverse_scale(sl.st->scale_cur);
    const int ie = pow2_exponent(isc);
    const int g = d.g;
    const int i = item.bx * BBX + threadIdx.x + g;
    const int j = item.by * BBY + threadIdx.y + g;
    if (i >= g + d.ni() || j >= g + d.nj()) continue;
    const int k0 = item.bz * lv.zc + g, k1 = min(k0 + lv.zc, g + d.nk());
    const float* e = (const float*)lv.phi;
    double* phi = sl.phi64;
    for (int k = k0; k < k1; k++) {
      const long long q = d.at(i, j, k);
      if (ie != INT_MIN) phi[q] += f32_to_f64_pow2(e[q], ie);
      else phi[q] = fma((double)e[q], isc, phi[q]);
    }
  }
}

// FP64 outer residual of the refinement (as k_delta in its refinement mode):
// stores the scaled FP32 inner right-hand side, one {sum, max} partial per tile.
template <int G>
__global__ void __launch_bounds__(BBX* BBY) kb_delta_ir(BArgs a, int list) {
  __shared__ double sh[64];
  const BList L = a.lists[list];
  const int tid = threadIdx.x + BBX * threadIdx.y;
  for (int it = blockIdx.x; it < L.total; it += gridDim.x) {
    const BTile item = find_tile(a.items, L, it);
    const BSlot& sl = a.slots[item.slot];
    if (sl.st->done) continue;   // uniform over the block
    const BLevel& lv = sl.lv[0];
    const Dims d = lv.d;
    const double oscale = sl.st->scale_next;
    const int oexp = pow2_exponent(oscale);
    const int i = item.bx * BBX + threadIdx.x + G;
    const int j = item.by * BBY + threadIdx.y + G;
    const int k0 = item.bz * lv.zc + G, k1 = min(k0 + lv.zc, G + d.nk());
    const long long sy = d.sy(), sz = d.sz();
    const double* phi = sl.phi64;
    const double* fs = sl.fs64;
    float* out = (float*)lv.fs;
    float s2f = 0.0f, mxf = 0.0f;
    if (i < G + d.ni() && j < G + d.nj()) {
      for (int k = k0; k < k1; k++) {
        const long long q = d.at(i, j, k);
        const double dd = gs_any<G>(lv.iso, phi, q, sy, sz, sl.cf0, fs[q]) - phi[q];
        const float v = oexp != INT_MIN ? f64_to_f32_pow2(dd, oexp) : (float)(dd * oscale);
        s2f = fmaf(v, v, s2f);
        mxf = fmaxf(mxf, fabsf(v));
        out[q] = v;
      }
    }
    // FP32 warp sums of the scaled values, unscaled once per warp, FP64 across warps
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s2f += __shfl_xor_sync(0xffffffffu, s2f, o);
      mxf = fmaxf(mxf, __shfl_xor_sync(0xffffffffu, mxf, o));
    }
    if ((tid & 31) == 0) {
      const double inv = inverse_scale(oscale);
      sh[tid >> 5] = (double)s2f * inv * inv;
      sh[32 + (tid >> 5)] = (double)mxf * inv;
    }
    __syncthreads();
    if (tid < 32) {
      double u = tid < 8 ? sh[tid] : 0.0, m = tid < 8 ? sh[32 + tid] : 0.0;
      u = warp_sum(u);
      m = warp_max(m);
      if (tid == 0) {
        sl.partials[2 * item.local] = u;
        sl.partials[2 * item.local + 1] = m;
      }
    }
    __syncthreads();
  }
}

__global__ void kb_gather(const BSlot* slots, int capacity, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= capacity) return;
  const BSlot& sl = slots[i];
  if (!sl.active) {
    out[2 * i] = -1;
    out[2 * i + 1] = 0;
    return;
  }
  out[2 * i] = sl.st->done;
  out[2 * i + 1] = sl.st->iter;
}

// ------------------------------------------------------------------ launchers
static const dim3 kTile(BBX, BBY);

cudaError_t launch_b_sweep(const BArgs& a, int order, int dt, int list, int colour, cudaStream_t s) {
  if (order == 2) {
    if (dt == DT_F64) kb_sweep<1, double><<<bgrid(), kTile, 0, s>>>(a, list, colour);
    else kb_sweep<1, float><<<bgrid(), kTile, 0, s>>>(a, list, colour);
  } else {
    if (dt == DT_F64) kb_sweep<2, double><<<bgrid(), kTile, 0, s>>>(a, list, colour);
    else kb_sweep<2, float><<<bgrid(), kTile, 0, s>>>(a, list, colour);
  }
  return cudaGetLastError();
}

cudaError_t launch_b_delta_skip(const BArgs& a, int order, int dt, int list, cudaStream_t s) {
  if (order == 2) {
    if (dt == DT_F64) kb_delta_skip<1, double><<<bgrid(), kTile, 0, s>>>(a, list);
    else kb_delta_skip<1, float><<<bgrid(), kTile, 0, s>>>(a, list);
  } else {
    if (dt == DT_F64) kb_delta_skip<2, double><<<bgrid(), kTile, 0, s>>>(a, list);
    else kb_delta_skip<2, float><<<bgrid(), kTile, 0, s>>>(a, list);
  }
  return cudaGetLastError();
}

cudaError_t launch_b_restrict(const BArgs& a, int dt, int list, cudaStream_t s) {
  if (dt == DT_F64) kb_restrict<double><<<bgrid(), kTile, 0, s>>>(a, list);
  else kb_restrict<float><<<bgrid(), kTile, 0, s>>>(a, list);
  return cudaGetLastError();
}

cudaError_t launch_b_prolong(const BArgs& a, int dt, int list, cudaStream_t s) {
  if (dt == DT_F64) kb_prolong<double><<<bgrid(), kTile, 0, s>>>(a, list);
  else kb_prolong<float><<<bgrid(), kTile, 0, s>>>(a, list);
  return cudaGetLastError();
}

template <int G, typename T>
static cudaError_t coarse_launch(const BArgs& a, int list, int max_blocks, size_t smem, double tol,
                                 cudaStream_t s) {
  auto kern = kb_coarse<G, T>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<max_blocks, 256, smem, s>>>(a, list, tol);
  return cudaGetLastError();
}

cudaError_t launch_b_coarse(const BArgs& a, int order, int dt, int list, int max_blocks,
                            size_t smem, double tol, cudaStream_t s) {
  if (order == 2)
    return dt == DT_F64 ? coarse_launch<1, double>(a, list, max_blocks, smem, tol, s)
                        : coarse_launch<1, float>(a, list, max_blocks, smem, tol, s);
  return dt == DT_F64 ? coarse_launch<2, double>(a, list, max_blocks, smem, tol, s)
                      : coarse_launch<2, float>(a, list, max_blocks, smem, tol, s);
}

cudaError_t launch_b_norm(const BArgs& a, int order, int list, cudaStream_t s) {
  if (order == 2) kb_norm<1><<<bgrid(), kTile, 0, s>>>(a, list);
  else kb_norm<2><<<bgrid(), kTile, 0, s>>>(a, list);
  return cudaGetLastError();
}

cudaError_t launch_b_finish(const BArgs& a, int list, int max_blocks, cudaStream_t s) {
  kb_finish<<<max_blocks, 1024, 0, s>>>(a, list);
  return cudaGetLastError();
}

cudaError_t launch_b_zero(const BArgs& a, int dt, int list, cudaStream_t s) {
  if (dt == DT_F64) kb_zero<double><<<bgrid(), kTile, 0, s>>>(a, list);
  else kb_zero<float><<<bgrid(), kTile, 0, s>>>(a, list);
  return cudaGetLastError();
}

cudaError_t launch_b_correct(const BArgs& a, int list, cudaStream_t s) {
  kb_correct<<<bgrid(), kTile, 0, s>>>(a, list);
  return cudaGetLastError();
}

cudaError_t launch_b_delta_ir(const BArgs& a, int order, int list, cudaStream_t s) {
  if (order == 2) kb_delta_ir<1><<<bgrid(), kTile, 0, s>>>(a, list);
  else kb_delta_ir<2><<<bgrid(), kTile, 0, s>>>(a, list);
  return cudaGetLastError();
}

cudaError_t launch_b_gather(const BSlot* slots, int capacity, int* out, cudaStream_t s) {
  kb_gather<<<(capacity + 127) / 128, 128, 0, s>>>(slots, capacity, out);
  return cudaGetLastError();
}

int batch_kernels_per_iteration(int nlev_max, int order, int prec, int nu1, int nu2, int inner) {
  const int ncol = order == 2 ? 2 : 3;
  const int down = nu1 * ncol + 3;   // sweeps, residual, restriction, coarsest CG
  const int up = 1 + nu2 * ncol;     // prolongation, sweeps
  const int vcycle = (nlev_max - 1) * (down + up);
  if (prec == 0) return vcycle + 2;            // + norm, finisher
  return 1 + inner * vcycle + 3;               // zero, cycles, correct, residual, finisher
}

}  // namespace ps
