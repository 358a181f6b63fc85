// TMA-staged z-marching tile kernels of the GB300 Poisson library.
//
// Both kernels walk a z-chunk of planes per thread block.  A ring of NS plane
// buffers in shared memory is filled by TMA boxes (cp.async.bulk.tensor, one
// mbarrier per stage) several planes ahead of the plane being computed, so the
// HBM stream never waits on the arithmetic.  Every array they read is a
// library-layout level array (rows padded to 32 elements).
//
// k_rb_sweep: one whole red-black Gauss-Seidel sweep of the 7-point operator
//   (Sec. 2.1.1, red = (i+j+k) even first), out of place.  Each warp marches a
//   strip of rows with the red values of three planes in registers; red values
//   just outside a strip or tile are recomputed from the same operands with the
//   same arithmetic, so the result is the sequential red-then-black sweep bit
//   for bit, while HBM traffic is one read of phi and fs and one write of phi
//   per sweep instead of per colour.
//
// k_resid_restrict: the fine residual delta = phi_GS - phi of each plane is
//   computed into shared memory on the tile's (2T+1)^2 footprint and folded at
//   once into the full-weighting sums of the coarse nodes (Sec. 2.1.3); the
//   fine residual never reaches HBM.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "tiled_kernels.cuh"
#include "tma.cuh"

namespace ps {

// ------------------------------------------------------------------ tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool encode_level_map(CUtensorMap* map, int dt, const void* base, const Dims& d, int bx, int by) {
  auto fn = encode_fn();
  if (!fn) return false;
  const size_t es = dt == DT_F64 ? 8 : dt == DT_F32 ? 4 : 2;
  const CUtensorMapDataType ty = dt == DT_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : dt == DT_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (((size_t)d.px * es) % 16 != 0 || ((uintptr_t)base & 15) != 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)d.ex, (cuuint64_t)d.ey, (cuuint64_t)d.ez};
  cuuint64_t strides[2] = {(cuuint64_t)d.px * es, (cuuint64_t)d.px * d.ey * es};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = fn(map, ty, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int sm_count() { return device_sm_count(); }

static constexpr int NT = 256;   // threads per block of both tile kernels

// x halo of a staged box: at least 2 nodes and a whole 16-byte TMA granule
template <typename T>
__host__ __device__ constexpr int xhalo() {
  return sizeof(T) >= 8 ? 2 : (int)(16 / sizeof(T));
}

// ================================================================== red-black sweep
// Register-blocked z-march.  Block = NWC warps over a 64 x TY tile (TY = R NWC);
// warp w owns the R grid rows ys .. ys+R-1 (ys = y0 + w R), lane l the x pair
// (xa, xa+1), xa = x0 + 2l, of which exactly one node is red on every row and
// plane: with ys and xa even, row r of plane p has its red node at xa + ((r+p)&1).
// Each step k of the march
//   * computes red(k+1) on rows -1 .. R of the strip (the two outer rows repeat
//     the neighbouring strips' arithmetic, so no warp waits for another's reds)
//     from the plane k+1 pairs held in registers, the plane k+2 pairs it loads
//     from the staged ring, and the old value of plane k kept from the last step;
//   * computes the red value of plane k+1 at the x-halo column of each row
//     (x0 - 1 or x0 + 64, whichever is red), lanes 0 .. R-1 one row each;
//   * finishes black(k) on rows 0 .. R-1 from the reds of planes k-1, k, k+1
//     (in-plane x neighbours from the adjacent lane by shuffle, the tile edges from
//     the halo reds) and stores the (red, black) pair of plane k.
// Every value repeats the colour passes' arithmetic on the same operands, so the
// result equals the sequential red-then-black sweep bit for bit.  Shared memory
// holds only the TMA ring of phi and fs planes; one barrier per plane releases
// the oldest stage to the next copy.
template <typename T, int R, int NWC, int NS>
struct SweepGeom {
  static_assert(R % 2 == 0, "rows per warp must be even (red column parity)");
  static constexpr int TX = 64;
  static constexpr int TY = R * NWC;
  static constexpr int NTH = 32 * NWC;
  static constexpr int XH = xhalo<T>();
  static constexpr int WP = TX + 2 * XH;           // staged row width (phi and fs)
  static constexpr int HP = TY + 4;                // phi rows: y0-2 .. y0+TY+1
  static constexpr int HF = TY + 2;                // fs rows:  y0-1 .. y0+TY
  static constexpr int PBYTES = WP * HP * (int)sizeof(T);
  static constexpr int FBYTES = WP * HF * (int)sizeof(T);
  static constexpr int PB = align_up(PBYTES, 128), FB = align_up(FBYTES, 128);
  static constexpr int SMEM = NS * (PB + FB) + NS * 8;
};

// two adjacent staged values as floats (the pair is 2-element aligned)
template <typename T> __device__ __forceinline__ float2 ld_pair(const T* p);
template <> __device__ __forceinline__ float2 ld_pair<float>(const float* p) {
  return *reinterpret_cast<const float2*>(p);
}
template <> __device__ __forceinline__ float2 ld_pair<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}
__device__ __forceinline__ float pick(float2 v, int c) { return c ? v.y : v.x; }

template <bool ISO>
__device__ __forceinline__ float gs7(float ax, float ay, float az, float f, const Coef<float>& cf) {
  if (ISO) return fma((ax + ay) + az, cf.c1[0], f);
  return fma(ax, cf.c1[0], fma(ay, cf.c1[1], fma(az, cf.c1[2], f)));
}

// Per-thread state of the march and one step of it (KP = parity of plane k).
template <typename T, bool ISO, int R, int NWC, int NS>
struct RbMarch {
  using S = St<T>;
  using Gm = SweepGeom<T, R, NWC, NS>;
  static constexpr int WP = Gm::WP;
  static constexpr int NR = R + 2;   // red rows -1 .. R   (index i = r + 1)
  static constexpr int NP = R + 4;   // phi rows -2 .. R+1 (index i = r + 2)
  static constexpr int PBE = Gm::PB / (int)sizeof(T), FBE = Gm::FB / (int)sizeof(T);
  static constexpr unsigned FULL = 0xffffffffu;

  const T* Pst;
  const T* Fst;
  unsigned long long* bar;
  Coef<float> cf;
  int l, x0, nx, nz, ny, ys, z0, pofs, hbase, hfbase;
  unsigned bm0, bm1;      // boundary bits of the red rows, per red column parity
  bool col_a, col_b, h_rowb;
  T* o;                   // output of (xa, ys) on the next black plane
  long long osz, opy;
  // pipeline
  bool ok;
  int wq, qk, qk1, qk2;
  unsigned wph;
  // registers carried from step to step
  float zlo[NR];          // phi(k) at the red column of plane k+1
  float rm[R], r0[NR], rp[NR];   // red(k-1) (rows 0..R-1), red(k), red(k+1)
  float fb[R];            // fs(k) at the black column
  float hk, hk1;          // halo reds of planes k, k+1 (lane l < R: row l)

  __device__ __forceinline__ void wait_next() {
    mbar_wait(&bar[wq], wph, ok);
    if (++wq == NS) { wq = 0; wph ^= 1u; }
  }

  template <int KP>
  __device__ __forceinline__ void step(int k, float2 (&A)[NP], float2 (&B)[NP]) {
    constexpr int PR = KP ^ 1;   // parity of plane k + 1
    wait_next();                 // plane k + 2
    const T* P0 = Pst + qk * PBE;
    const T* P1 = Pst + qk1 * PBE;
    const T* P2 = Pst + qk2 * PBE;
    const T* F1 = Fst + qk1 * FBE;
#pragma unroll
    for (int i = 0; i < NP; i++) B[i] = ld_pair(P2 + pofs + i * WP);
    float2 ff[NR];
#pragma unroll
    for (int i = 0; i < NR; i++) ff[i] = ld_pair(F1 + pofs + i * WP);
    const bool pb = k + 1 <= 0 || k + 1 >= nz;
    // red(k+1), rows -1 .. R
#pragma unroll
    for (int i = 0; i < NR; i++) {
      const int c = (i + 1 + PR) & 1;   // red column of row i-1 (compile-time)
      const float2 a = A[i + 1];
      float nb;
      if (c == 0) {
        nb = __shfl_up_sync(FULL, a.y, 1);
        if (l == 0) nb = S::ld(P1 + pofs + (i + 1) * WP - 1);
      } else {
        nb = __shfl_down_sync(FULL, a.x, 1);
        if (l == 31) nb = S::ld(P1 + pofs + (i + 1) * WP + 2);
      }
      const float ax = nb + (c ? a.x : a.y);
      const float ay = pick(A[i], c) + pick(A[i + 2], c);
      const float az = pick(B[i + 1], c) + zlo[i];
      const float v = gs7<ISO>(ax, ay, az, pick(ff[i], c), cf);
      const bool bnd = pb || (((c ? bm1 : bm0) >> i) & 1u);
      rp[i] = stored<T>(bnd ? pick(a, c) : v);
    }
    // halo red(k+1) of row l (lanes 0 .. R-1)
    if (l < R) {
      const int c = (l + PR) & 1;
      const int hc = c ? -1 : Gm::TX;   // x0 - 1 is red where the pair's red is odd
      const int pi = hbase + hc;
      const float ax = S::ld(P1 + pi + 1) + S::ld(P1 + pi - 1);
      const float ay = S::ld(P1 + pi + WP) + S::ld(P1 + pi - WP);
      const float az = S::ld(P2 + pi) + S::ld(P0 + pi);
      const float v = gs7<ISO>(ax, ay, az, S::ld(F1 + hfbase + hc), cf);
      const int hx = x0 + hc;
      const bool bnd = pb || h_rowb || hx <= 0 || hx >= nx;
      hk1 = stored<T>(bnd ? S::ld(P1 + pi) : v);
    }
    // black(k), rows 0 .. R-1, and the store of plane k
    if (k >= z0) {
#pragma unroll
      for (int r = 0; r < R; r++) {
        const int cb = (r + KP + 1) & 1;   // black column on plane k
        const float own = r0[r + 1];       // red(k) in the pair
        const float hv = __shfl_sync(FULL, hk, r);
        float nb;
        if (cb == 0) {
          nb = __shfl_up_sync(FULL, own, 1);
          if (l == 0) nb = hv;
        } else {
          nb = __shfl_down_sync(FULL, own, 1);
          if (l == 31) nb = hv;
        }
        const float ax = nb + own;
        const float ay = r0[r] + r0[r + 2];
        const float az = rp[r + 1] + rm[r];
        const float vb = gs7<ISO>(ax, ay, az, fb[r], cf);
        const float v0 = cb ? own : vb, v1 = cb ? vb : own;
        const int yy = ys + r;
        if (yy >= 1 && yy < ny) {
          T* orow = o + r * opy;
          if (col_a && col_b) {
            St2<T>::st(orow, v0, v1);
          } else {
            if (col_a) S::st(orow, v0);
            if (col_b) S::st(orow + 1, v1);
          }
        }
      }
      o += osz;
    }
    // carry to step k + 1
#pragma unroll
    for (int r = 0; r < R; r++) rm[r] = r0[r + 1];
#pragma unroll
    for (int i = 0; i < NR; i++) {
      r0[i] = rp[i];
      zlo[i] = pick(A[i + 1], (i + 1 + KP) & 1);   // phi(k+1) at the red column of plane k+2
    }
#pragma unroll
    for (int r = 0; r < R; r++) fb[r] = pick(ff[r + 1], ((r + PR) & 1) ^ 1);
    hk = hk1;
  }
};

template <typename T, bool ISO, int R, int NWC, int NS>
__global__ void __launch_bounds__(32 * NWC)
    k_rb_sweep(const __grid_constant__ CUtensorMap mP, const __grid_constant__ CUtensorMap mF, Dims d,
               Coef<float> cf, T* __restrict__ out, int zc, const DevState* __restrict__ st,
               int* __restrict__ fault) {
  using S = St<T>;
  using Gm = SweepGeom<T, R, NWC, NS>;
  using M = RbMarch<T, ISO, R, NWC, NS>;
  constexpr int WP = Gm::WP, XH = Gm::XH, NR = M::NR, NP = M::NP, PBE = M::PBE, FBE = M::FBE;
  extern __shared__ __align__(128) unsigned char smem[];
  T* Pst = reinterpret_cast<T*>(smem);
  T* Fst = reinterpret_cast<T*>(smem + NS * Gm::PB);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + NS * (Gm::PB + Gm::FB));

  if (st != nullptr && st->done) return;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int nx = d.nx, ny = d.ny, nz = d.nz;
  const int x0 = blockIdx.x * Gm::TX, y0 = blockIdx.y * Gm::TY;
  const int z0 = 1 + blockIdx.z * zc;   // zc is even: z0 is odd in every block
  const int z1 = min(z0 + zc, nz);      // output planes [z0, z1)
  const int zl = z0 - 2, zh = z1 + 1;   // staged planes [zl, zh]
  if (tid == 0) {
    for (int q = 0; q < NS; q++) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int z, int q) {   // thread 0: stage q <- plane z
    if (z > zh) return;
    mbar_expect_tx(&bar[q], Gm::PBYTES + Gm::FBYTES);
    tma_load_3d(Pst + q * PBE, &mP, x0 - XH, y0 - 2, z, &bar[q]);
    tma_load_3d(Fst + q * FBE, &mF, x0 - XH, y0 - 1, z, &bar[q]);
  };
  if (tid == 0)
    for (int q = 0; q < NS; q++) issue(zl + q, q);

  M m;
  m.Pst = Pst;
  m.Fst = Fst;
  m.bar = bar;
  m.cf = cf;
  m.l = l;
  m.x0 = x0;
  m.nx = nx;
  m.ny = ny;
  m.nz = nz;
  m.ys = y0 + w * R;
  m.z0 = z0;
  const int xa = x0 + 2 * l;
  const int prow = w * R * WP + XH;   // staged phi row of grid row ys-2 / fs row of ys-1, at x0
  m.pofs = prow + 2 * l;
  unsigned rowb = 0;
#pragma unroll
  for (int i = 0; i < NR; i++)
    if (m.ys + i - 1 <= 0 || m.ys + i - 1 >= ny) rowb |= 1u << i;
  m.bm0 = (xa <= 0 || xa >= nx) ? ~0u : rowb;
  m.bm1 = (xa + 1 >= nx) ? ~0u : rowb;
  m.col_a = xa >= 1 && xa < nx;
  m.col_b = xa + 1 < nx;
  m.h_rowb = m.ys + l <= 0 || m.ys + l >= ny;
  m.hbase = prow + (l + 2) * WP;
  m.hfbase = prow + (l + 1) * WP;
  m.o = out + ((long long)z0 * d.ey + m.ys) * d.px + xa;
  m.osz = d.sz();
  m.opy = d.px;
  m.ok = true;
  m.wq = 0;
  m.wph = 0;
  m.hk = m.hk1 = 0.f;
#pragma unroll
  for (int i = 0; i < R; i++) m.rm[i] = m.fb[i] = 0.f;
#pragma unroll
  for (int i = 0; i < NR; i++) m.r0[i] = 0.f;

  // prologue: phi(zl) at the red column of plane zl+1 (zl is odd: parity 0), pairs of plane zl+1
  float2 PA[NP], PB2[NP];   // phi pairs of planes k+1 and k+2 (roles alternate by step)
  m.wait_next();
  m.wait_next();
#pragma unroll
  for (int i = 0; i < NR; i++) m.zlo[i] = S::ld(Pst + m.pofs + (i + 1) * WP + ((i + 1) & 1));
#pragma unroll
  for (int i = 0; i < NP; i++) PA[i] = ld_pair(Pst + PBE + m.pofs + i * WP);
  m.qk = 0;
  m.qk1 = 1;
  m.qk2 = 2 % NS;
  auto release = [&](int k) {   // the stage of plane k takes plane k + NS
    __syncthreads();
    if (tid == 0 && m.ok) {   // after a failed wait no new copy is issued
      fence_proxy_async();
      issue(k + NS, m.qk);
    }
    m.qk = m.qk1;
    m.qk1 = m.qk2;
    m.qk2 = m.qk2 + 1 == NS ? 0 : m.qk2 + 1;
  };
  for (int k = zl; k < z1; k += 2) {
    m.template step<1>(k, PA, PB2);   // zl is odd
    release(k);
    if (k + 1 < z1) {
      m.template step<0>(k + 1, PB2, PA);
      release(k + 1);
    }
  }
  if (!m.ok && fault != nullptr) atomicExch(fault, 1);
}

template <typename T, bool ISO, int R, int NWC>
static cudaError_t rb_sweep_t(const Dims& d, const double h[3], const void* pin, void* pout,
                              const void* fs, const DevState* st, int* fault, cudaStream_t s) {
  constexpr int NS = 5;
  using Gm = SweepGeom<T, R, NWC, NS>;
  auto kern = k_rb_sweep<T, ISO, R, NWC, NS>;
  static int blocks_per_sm = 0;
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, Gm::NTH, Gm::SMEM);
    if (e != cudaSuccess) return e;
    blocks_per_sm = std::max(1, blocks_per_sm);
  }
  const int dt = sizeof(T) == 4 ? DT_F32 : DT_BF16;
  CUtensorMap mP, mF;
  if (!encode_level_map(&mP, dt, pin, d, Gm::WP, Gm::HP) || !encode_level_map(&mF, dt, fs, d, Gm::WP, Gm::HF))
    return cudaErrorInvalidValue;
  const int gx = (d.nx - 1) / Gm::TX + 1, gy = (d.ny - 1) / Gm::TY + 1;
  const int nk = d.nz - 1;
  // one wave: as many z-chunks per tile column as keep every block resident;
  // chunks hold an even number of planes (every chunk starts on an odd plane)
  const int slots = sm_count() * blocks_per_sm;
  const int nchunk = std::max(1, std::min(nk, slots / (gx * gy)));
  int zc = (nk + nchunk - 1) / nchunk;
  zc += zc & 1;
  const dim3 grid(gx, gy, (nk + zc - 1) / zc);
  const Coef<float> cf = make_coef<float>(d, h, 2);
  kern<<<grid, Gm::NTH, Gm::SMEM, s>>>(mP, mF, d, cf, (T*)pout, zc, st, fault);
  return cudaGetLastError();
}

template <typename T, int R, int NWC>
static cudaError_t rb_sweep_iso(const Dims& d, const double h[3], const void* pin, void* pout,
                                const void* fs, const DevState* st, int* fault, cudaStream_t s) {
  if (h[0] == h[1] && h[1] == h[2]) return rb_sweep_t<T, true, R, NWC>(d, h, pin, pout, fs, st, fault, s);
  return rb_sweep_t<T, false, R, NWC>(d, h, pin, pout, fs, st, fault, s);
}

// Tile variants (rows per warp x warps per block; 64 columns, 5-stage ring):
// 1 = 4 x 4 (64 x 16 tile), 2 = 2 x 4 (64 x 8), 3 = 8 x 4 (64 x 32),
// 4 = 4 x 8 (64 x 32).  0 picks the storage type's default: 1 for FP32, 3 for
// BF16 (measured at 256^3 among 2-8 rows, 4-8 warps and 4-6 stages: 0.043 ms
// FP32, 0.033 ms BF16).  The autotuner chooses among them per grid.
int rb_sweep_default_tile(int dt) { return dt == DT_F32 ? 1 : 3; }

template <typename T>
static cudaError_t rb_sweep_dispatch(const Dims& d, const double h[3], const void* pin, void* pout,
                                     const void* fs, const DevState* st, int* fault, int tile, cudaStream_t s) {
  switch (tile) {
    case 1: return rb_sweep_iso<T, 4, 4>(d, h, pin, pout, fs, st, fault, s);
    case 2: return rb_sweep_iso<T, 2, 4>(d, h, pin, pout, fs, st, fault, s);
    case 3: return rb_sweep_iso<T, 8, 4>(d, h, pin, pout, fs, st, fault, s);
    case 4: return rb_sweep_iso<T, 4, 8>(d, h, pin, pout, fs, st, fault, s);
    default: return cudaErrorInvalidValue;
  }
}

// FP64 levels keep the colour passes (their sweeps are bound by the FP64 pipe),
// so the fused sweep is built for the FP32 and BF16 inner levels only.
cudaError_t launch_rb_sweep(const Dims& d, int order, const double h[3], int dt, const void* phi_in,
                            void* phi_out, const void* fs, const DevState* st, int* fault,
                            cudaStream_t s, int tile) {
  if (order != 2 || d.g != 1 || dt == DT_F64) return cudaErrorNotSupported;
  if (tile < 0 || tile > kRbSweepTiles) return cudaErrorInvalidValue;
  if (tile == 0) tile = rb_sweep_default_tile(dt);
  if (dt == DT_F32) return rb_sweep_dispatch<float>(d, h, phi_in, phi_out, fs, st, fault, tile, s);
  return rb_sweep_dispatch<__nv_bfloat16>(d, h, phi_in, phi_out, fs, st, fault, tile, s);
}

// ================================================================== residual + restriction
// Coarse tile TXC x TYC; the fine residual footprint is (2 TXC + 1) x (2 TYC + 1).
template <typename T, int G, int TXC, int TYC>
struct RRGeom {
  static constexpr int XA = xhalo<T>();                           // box starts XA before 2 I0
  static constexpr int AL = (int)(16 / sizeof(T)) > 0 ? (int)(16 / sizeof(T)) : 1;
  static constexpr int WP = align_up(2 * TXC + 2 * G - 1 + XA, AL);   // staged row width
  static constexpr int HP = 2 * TYC + 2 * G + 1;                     // phi rows
  static constexpr int HF = 2 * TYC + 1;                             // fs rows
  static constexpr int DW = 2 * TXC + 1, DH = 2 * TYC + 1;           // residual footprint
  static constexpr int NS = 2 * G + 3;                               // phi planes in the ring
  static constexpr int PBYTES = WP * HP * (int)sizeof(T);
  static constexpr int FBYTES = WP * HF * (int)sizeof(T);
  static constexpr int PB = align_up(PBYTES, 128), FB = align_up(FBYTES, 128);
};

template <typename TF, typename TC, int G, bool ISO, int TXC, int TYC>
__global__ void __launch_bounds__(NT)
    k_resid_restrict(const __grid_constant__ CUtensorMap mP, const __grid_constant__ CUtensorMap mF,
                     Dims fd, Dims cd, Coef<typename St<TF>::C> cf, TC* __restrict__ fsc,
                     typename St<TF>::C sc, int kc, int* __restrict__ fault) {
  using C = typename St<TF>::C;
  using S = St<TF>;
  using Gm = RRGeom<TF, G, TXC, TYC>;
  constexpr int NS = Gm::NS, WP = Gm::WP, DW = Gm::DW, DH = Gm::DH;
  constexpr int PBE = Gm::PB / (int)sizeof(TF), FBE = Gm::FB / (int)sizeof(TF);
  extern __shared__ __align__(128) unsigned char smem[];
  TF* Pst = reinterpret_cast<TF*>(smem);
  TF* Fst = reinterpret_cast<TF*>(smem + NS * Gm::PB);
  C* D = reinterpret_cast<C*>(smem + NS * (Gm::PB + Gm::FB));
  unsigned long long* bar =
      reinterpret_cast<unsigned long long*>(smem + NS * (Gm::PB + Gm::FB) + align_up(DW * DH * (int)sizeof(C), 128));

  const int tid = threadIdx.x;
  const int I0 = blockIdx.x * TXC, J0 = blockIdx.y * TYC;   // coarse nodes of the tile
  const int K0 = 1 + blockIdx.z * kc;
  const int K1 = min(K0 + kc, cd.nz);                        // coarse planes [K0, K1)
  const int nfx = fd.nx, nfy = fd.ny, nfz = fd.nz;
  // array coordinates (node + G - 1) of the staged boxes
  const int bxs = 2 * I0 - Gm::XA;
  const int bys = 2 * J0 - 2;          // phi rows
  const int byf = 2 * J0 + G - 2;      // fs rows
  const int pz_lo = 2 * K0 - 2, pz_hi = 2 * K1 + 2 * G - 2;   // phi planes staged
  const int pc_lo = 2 * K0 + G - 2, pc_hi = 2 * K1 + G - 2;   // residual planes (array index)
  if (tid == 0) {
    for (int q = 0; q < NS; q++) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // stage of phi plane pz also carries fs plane pz - G when that is a residual plane
  auto issue = [&](int pz) {
    if (pz > pz_hi) return;
    const int q = (pz - pz_lo) % NS;
    const bool withf = pz - G >= pc_lo;
    mbar_expect_tx(&bar[q], Gm::PBYTES + (withf ? Gm::FBYTES : 0));
    tma_load_3d(Pst + q * PBE, &mP, bxs, bys, pz, &bar[q]);
    if (withf) tma_load_3d(Fst + q * FBE, &mF, bxs, byf, pz - G, &bar[q]);
  };
  bool ok = true;
  int next_wait = pz_lo;
  auto wait_upto = [&](int pz) {
    for (; next_wait <= pz; next_wait++) {
      const int u = next_wait - pz_lo;
      mbar_wait(&bar[u % NS], (unsigned)((u / NS) & 1), ok);
    }
  };
  if (tid == 0)
    for (int pz = pz_lo; pz < pz_lo + NS; pz++) issue(pz);

  // this thread's residual nodes of the footprint (fixed for every plane): staged phi
  // offset, fs offset, footprint index, and whether the node is interior in x and y
  constexpr int NFP = DW * DH;
  constexpr int PERD = (NFP + NT - 1) / NT;
  int pp_e[PERD], ff_e[PERD];
  bool in_e[PERD];
#pragma unroll
  for (int e = 0; e < PERD; e++) {
    const int idx = tid + e * NT;
    const int r = idx / DW, c = idx - r * DW;
    const int fx = 2 * I0 - 1 + c, fy = 2 * J0 - 1 + r;   // fine nodes
    const int col = fx + G - 1 - bxs;
    pp_e[e] = (fy + G - 1 - bys) * WP + col;
    ff_e[e] = (fy + G - 1 - byf) * WP + col;
    in_e[e] = idx < NFP && fx >= 1 && fx < nfx && fy >= 1 && fy < nfy;
  }
  // this thread's coarse nodes (in-tile index t, t + NT, ...)
  constexpr int NCT = TXC * TYC;
  constexpr int PER = (NCT + NT - 1) / NT;
  C pm[PER], p0[PER];
#pragma unroll
  for (int e = 0; e < PER; e++) { pm[e] = (C)0; p0[e] = (C)0; }
  auto wrap = [](int q) { return q >= NS ? q - NS : (q < 0 ? q + NS : q); };

  int qc = G;   // stage of residual plane pc: phi plane pc sits in stage (pc - pz_lo) % NS, pc_lo - pz_lo = G
  for (int pc = pc_lo; pc <= pc_hi; pc++) {
    wait_upto(pc + G);
    const int fz = pc - G + 1;   // fine node index of this residual plane
    const bool zin = fz >= 1 && fz < nfz;
    const TF* Pc = Pst + qc * PBE;
    const TF* Pz1p = Pst + wrap(qc + 1) * PBE;
    const TF* Pz1m = Pst + wrap(qc - 1) * PBE;
    const TF* Pz2p = Pst + wrap(qc + 2) * PBE;
    const TF* Pz2m = Pst + wrap(qc - 2) * PBE;
    const TF* F = Fst + wrap(qc + G) * FBE;
#pragma unroll
    for (int e = 0; e < PERD; e++) {
      const int idx = tid + e * NT;
      if (idx >= NFP) break;
      C dl = (C)0;
      if (zin && in_e[e]) {
        const int pp = pp_e[e];
        const C ax = S::ld(Pc + pp + 1) + S::ld(Pc + pp - 1);
        const C ay = S::ld(Pc + pp + WP) + S::ld(Pc + pp - WP);
        const C az = S::ld(Pz1p + pp) + S::ld(Pz1m + pp);
        const C f = S::ld(F + ff_e[e]);
        C v;
        if (ISO) v = fma((ax + ay) + az, cf.c1[0], f);
        else v = fma(ax, cf.c1[0], fma(ay, cf.c1[1], fma(az, cf.c1[2], f)));
        if (G == 2) {
          const C bx = S::ld(Pc + pp + 2) + S::ld(Pc + pp - 2);
          const C by = S::ld(Pc + pp + 2 * WP) + S::ld(Pc + pp - 2 * WP);
          const C bz = S::ld(Pz2p + pp) + S::ld(Pz2m + pp);
          if (ISO) v = fma((bx + by) + bz, cf.c2[0], v);
          else v = fma(bx, cf.c2[0], fma(by, cf.c2[1], fma(bz, cf.c2[2], v)));
        }
        dl = v - S::ld(Pc + pp);
      }
      D[idx] = dl;
    }
    __syncthreads();
    const bool odd = (fz & 1) != 0;
#pragma unroll
    for (int e = 0; e < PER; e++) {
      const int t = tid + e * NT;
      if (t >= NCT) break;
      const int li = t % TXC, lj = t / TXC;
      const C* d0 = D + (2 * lj) * DW + 2 * li;   // fine (2I-1, 2J-1)
      C rows[3];
#pragma unroll
      for (int dy = 0; dy < 3; dy++) {
        const C* q = d0 + dy * DW;
        rows[dy] = (q[0] + q[2]) + (C)2 * q[1];
      }
      const C plane = (rows[0] + rows[2]) + (C)2 * rows[1];
      if (!odd) {
        p0[e] = plane;
      } else {
        const int K = (fz - 1) / 2;   // fz = 2K + 1 closes coarse plane K
        const int I = I0 + li, J = J0 + lj;
        if (K >= K0 && I >= 1 && I < cd.nx && J >= 1 && J < cd.ny) {
          const C acc = (pm[e] + plane) + (C)2 * p0[e];
          St<TC>::st(fsc + cd.at(I + G - 1, J + G - 1, K + G - 1), (typename St<TC>::C)(acc * sc));
        }
        pm[e] = plane;
      }
    }
    __syncthreads();
    if (tid == 0 && ok) {   // after a failed wait no new copy is issued
      fence_proxy_async();
      issue(pc - G + NS);   // stage of phi plane pc - G
    }
    qc = wrap(qc + 1);
  }
  wait_upto(pz_hi);
  if (!ok && fault != nullptr) atomicExch(fault, 1);
}

// ------------------------------------------------------------------ register-blocked (7-point)
// The FP32/BF16 7-point levels use k_resid_restrict_rb; the shared-memory
// kernel above serves the 13-point operator and FP64 levels.

// Block = NWC warps over a tile of 32 x TYC coarse nodes (TYC = RC NWC), i.e.
// 64 fine columns.  Warp w owns the coarse rows Jw .. Jw+RC-1 (Jw = J0 + w RC)
// and the fine residual rows 2Jw-1 .. 2Jw+2RC-1 (ND = 2RC+1 rows: the last is
// also the first of the next strip and is computed by both); lane l owns the
// fine x pair (2I, 2I+1), I = I0 + l, i.e. coarse column I.  Each step of the
// z-march computes the residual of one fine plane z:
//   * phi of planes z-1 and z is held in registers (rows -1 .. ND of the
//     strip), plane z+1 is read from the staged ring, and the three roles
//     rotate through three register arrays from step to step;
//   * x neighbours come from the adjacent lane by shuffle (the tile's edge
//     columns from the staged plane), and lanes 0 .. ND-1 compute the residual
//     at x = 2 I0 - 1 (left of the tile) for row l+1, handed to lane 0;
//   * full weighting runs in registers: a row sum per fine row (the 2I-1 term
//     by shuffle), the (y-1, y, y+1) combination per coarse row, and the
//     (z-1, z, z+1) combination of carried plane sums when z closes a coarse
//     plane.
// The residual and every weighted sum are formed in the order of
// k_resid_restrict, so both kernels give the same coarse right-hand side bit
// for bit.
template <typename T, int RC, int NWC, int NS>
struct RrbGeom {
  static constexpr int TX = 64, TXC = 32, TYC = RC * NWC, NTH = 32 * NWC;
  static constexpr int ND = 2 * RC + 1;    // fine residual rows of a strip
  static constexpr int NPR = ND + 2;       // phi rows of a strip
  static constexpr int XH = xhalo<T>();    // >= 4 columns: covers x0 - 2
  static constexpr int WP = TX + 2 * XH;   // staged row width
  static constexpr int HP = 2 * TYC + 3;   // phi rows 2J0-2 .. 2J0+2TYC
  static constexpr int HF = 2 * TYC + 1;   // fs rows  2J0-1 .. 2J0+2TYC-1
  static constexpr int PBYTES = WP * HP * (int)sizeof(T), FBYTES = WP * HF * (int)sizeof(T);
  static constexpr int PB = align_up(PBYTES, 128), FB = align_up(FBYTES, 128);
  static constexpr int SMEM = NS * (PB + FB) + NS * 8;
};

template <typename T, bool ISO, int RC, int NWC, int NS>
struct RrbMarch {
  using S = St<T>;
  using Gm = RrbGeom<T, RC, NWC, NS>;
  static constexpr int WP = Gm::WP, ND = Gm::ND, NPR = Gm::NPR;
  static constexpr int PBE = Gm::PB / (int)sizeof(T), FBE = Gm::FB / (int)sizeof(T);
  static constexpr unsigned FULL = 0xffffffffu;

  const T* Pst;
  const T* Fst;
  unsigned long long* bar;
  Coef<float> cf;
  float sc;
  int l, pofs, hofs, hfofs, nfz, K0, K1, dir;
  unsigned rowin;    // bit i: fine row i of the strip (0 .. NPR-1) is interior
  bool ain, bin;     // the pair's nodes are interior in x
  bool hin;          // lane l < ND: the halo node (2 I0 - 1, row l + 1) is interior in x and y
  unsigned jok;      // bit j: coarse row Jw + j is interior; 0 if coarse column I is not
  float* o;          // coarse node (I, Jw, 0)
  long long cpy, cpz;
  bool ok;
  int wq, qm, q0, q1;
  unsigned wph;
  float pm[RC], p0[RC];   // plane sums of the last odd and the last even fine plane

  __device__ __forceinline__ void wait_next() {
    mbar_wait(&bar[wq], wph, ok);
    if (++wq == NS) { wq = 0; wph ^= 1u; }
  }

  // residual of fine plane z from Zm (the plane before z in the march), A
  // (plane z); Z1 <- the plane after z.  z -/+ 1 enter only as the sum
  // Z1 + Zm, the same value in either direction.
  __device__ __forceinline__ void step(int z, const float2 (&Zm)[NPR], const float2 (&A)[NPR], float2 (&Z1)[NPR]) {
    wait_next();   // plane z + dir (with fs of plane z)
    const T* Pm = Pst + qm * PBE;
    const T* P0 = Pst + q0 * PBE;
    const T* P1 = Pst + q1 * PBE;
    const T* F = Fst + q1 * FBE;
#pragma unroll
    for (int i = 0; i < NPR; i++) Z1[i] = ld_pair(P1 + pofs + i * WP);
    const bool zin = z >= 1 && z < nfz;
    // residual left of the tile, row l + 1 (lanes 0 .. ND-1)
    float hd = 0.f;
    if (l < ND) {
      const float ax = S::ld(P0 + hofs + 1) + S::ld(P0 + hofs - 1);
      const float ay = S::ld(P0 + hofs + WP) + S::ld(P0 + hofs - WP);
      const float az = S::ld(P1 + hofs) + S::ld(Pm + hofs);
      const float v = gs7<ISO>(ax, ay, az, S::ld(F + hfofs), cf);
      if (zin && hin) hd = v - S::ld(P0 + hofs);
    }
    float rs[ND];   // row sums of coarse column I, fine rows 1 .. ND
#pragma unroll
    for (int i = 1; i <= ND; i++) {
      const float2 a = A[i];
      float lf = __shfl_up_sync(FULL, a.y, 1);
      if (l == 0) lf = S::ld(P0 + pofs + i * WP - 1);
      float rt = __shfl_down_sync(FULL, a.x, 1);
      if (l == 31) rt = S::ld(P0 + pofs + i * WP + 2);
      const float2 f = ld_pair(F + pofs + (i - 1) * WP);
      const float va = gs7<ISO>(a.y + lf, A[i + 1].x + A[i - 1].x, Z1[i].x + Zm[i].x, f.x, cf);
      const float vb = gs7<ISO>(rt + a.x, A[i + 1].y + A[i - 1].y, Z1[i].y + Zm[i].y, f.y, cf);
      const bool rin = zin && ((rowin >> i) & 1u);
      const float da = rin && ain ? va - a.x : 0.f;
      const float db = rin && bin ? vb - a.y : 0.f;
      float nb = __shfl_up_sync(FULL, db, 1);
      const float hv = __shfl_sync(FULL, hd, i - 1);
      if (l == 0) nb = hv;
      rs[i - 1] = (nb + db) + 2.f * da;
    }
    if ((z & 1) == 0) {
#pragma unroll
      for (int j = 0; j < RC; j++) p0[j] = (rs[2 * j] + rs[2 * j + 2]) + 2.f * rs[2 * j + 1];
    } else {
      // odd z closes coarse plane K = (z - dir) / 2: its planes 2K -/+ 1 enter
      // as the sum pm + pl, the same value in either direction
      const int K = (z - dir) / 2;
#pragma unroll
      for (int j = 0; j < RC; j++) {
        const float pl = (rs[2 * j] + rs[2 * j + 2]) + 2.f * rs[2 * j + 1];
        if (K >= K0 && K < K1 && ((jok >> j) & 1u)) o[j * cpy + K * cpz] = ((pm[j] + pl) + 2.f * p0[j]) * sc;
        pm[j] = pl;
      }
    }
  }
};

// Blocks of odd z-chunks march down, even ones up: the fine planes two
// adjacent chunks both read are then read by both near the same time (both at
// the start or both at the end of their marches), so the second read hits L2.
template <typename T, bool ISO, int RC, int NWC, int NS>
__global__ void __launch_bounds__(32 * NWC, 2)
    k_resid_restrict_rb(const __grid_constant__ CUtensorMap mP, const __grid_constant__ CUtensorMap mF, Dims fd,
                        Dims cd, Coef<float> cf, float* __restrict__ fsc, float sc, int kc,
                        int* __restrict__ fault) {
  using Gm = RrbGeom<T, RC, NWC, NS>;
  using M = RrbMarch<T, ISO, RC, NWC, NS>;
  constexpr int WP = Gm::WP, XH = Gm::XH, ND = Gm::ND, NPR = Gm::NPR, PBE = M::PBE, FBE = M::FBE;
  extern __shared__ __align__(128) unsigned char smem[];
  T* Pst = reinterpret_cast<T*>(smem);
  T* Fst = reinterpret_cast<T*>(smem + NS * Gm::PB);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + NS * (Gm::PB + Gm::FB));

  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int I0 = blockIdx.x * Gm::TXC, J0 = blockIdx.y * Gm::TYC;
  const int K0 = 1 + blockIdx.z * kc;
  const int K1 = min(K0 + kc, cd.nz);   // coarse planes [K0, K1)
  const int x0 = 2 * I0;
  const int dir = (blockIdx.z & 1) ? -1 : 1;
  const int np = 2 * (K1 - K0) + 3;                // staged phi planes 2K0-2 .. 2K1, t = 0 .. np-1
  const int pfirst = dir > 0 ? 2 * K0 - 2 : 2 * K1;  // plane of t = 0
  if (tid == 0) {
    for (int q = 0; q < NS; q++) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // stage of the t-th phi plane p also carries fs of plane p - dir (t >= 2: a residual plane)
  auto issue = [&](int t) {
    if (t >= np) return;
    const int q = t % NS;
    const int p = pfirst + dir * t;
    const bool withf = t >= 2;
    mbar_expect_tx(&bar[q], Gm::PBYTES + (withf ? Gm::FBYTES : 0));
    tma_load_3d(Pst + q * PBE, &mP, x0 - XH, 2 * J0 - 2, p, &bar[q]);
    if (withf) tma_load_3d(Fst + q * FBE, &mF, x0 - XH, 2 * J0 - 1, p - dir, &bar[q]);
  };
  if (tid == 0)
    for (int t = 0; t < NS; t++) issue(t);

  M m;
  m.Pst = Pst;
  m.Fst = Fst;
  m.bar = bar;
  m.cf = cf;
  m.sc = sc;
  m.l = l;
  m.nfz = fd.nz;
  m.K0 = K0;
  m.K1 = K1;
  m.dir = dir;
  const int Jw = J0 + w * RC;
  const int y0 = 2 * Jw - 2;   // fine row of strip row 0
  const int brow = 2 * w * RC;  // staged phi row of strip row 0; staged fs row of strip row 1
  m.pofs = brow * WP + XH + 2 * l;
  m.hofs = (brow + l + 1) * WP + XH - 1;
  m.hfofs = (brow + l) * WP + XH - 1;
  unsigned rowin = 0;
#pragma unroll
  for (int i = 0; i < NPR; i++)
    if (y0 + i >= 1 && y0 + i < fd.ny) rowin |= 1u << i;
  m.rowin = rowin;
  const int xa = x0 + 2 * l;
  m.ain = xa >= 1 && xa < fd.nx;
  m.bin = xa + 1 < fd.nx;
  m.hin = l < ND && x0 - 1 >= 1 && ((rowin >> (l + 1)) & 1u);
  const int I = I0 + l;
  unsigned jok = 0;
  if (I >= 1 && I < cd.nx) {
#pragma unroll
    for (int j = 0; j < RC; j++)
      if (Jw + j >= 1 && Jw + j < cd.ny) jok |= 1u << j;
  }
  m.jok = jok;
  m.o = fsc + cd.at(min(I, cd.ex - 1), min(Jw, cd.ey - 1), 0);
  m.cpy = cd.sy();
  m.cpz = cd.sz();
  m.ok = true;
  m.wq = 0;
  m.wph = 0;
#pragma unroll
  for (int j = 0; j < RC; j++) m.pm[j] = m.p0[j] = 0.f;

  float2 X[NPR], Y[NPR], W[NPR];
  m.wait_next();   // t = 0
  m.wait_next();   // t = 1
#pragma unroll
  for (int i = 0; i < NPR; i++) {
    X[i] = ld_pair(Pst + m.pofs + i * WP);
    Y[i] = ld_pair(Pst + PBE + m.pofs + i * WP);
  }
  m.qm = 0;
  m.q0 = 1;
  m.q1 = 2 % NS;
  auto release = [&](int t) {   // the stage of plane t - 1 takes plane t - 1 + NS
    __syncthreads();
    if (tid == 0 && m.ok) {     // after a failed wait no new copy is issued
      fence_proxy_async();
      issue(t - 1 + NS);
    }
    m.qm = m.q0;
    m.q0 = m.q1;
    m.q1 = m.q1 + 1 == NS ? 0 : m.q1 + 1;
  };
  const int tl = np - 2;   // residual planes t = 1 .. np-2
  for (int t = 1; t <= tl; t += 3) {
    m.step(pfirst + dir * t, X, Y, W);
    release(t);
    if (t + 1 <= tl) {
      m.step(pfirst + dir * (t + 1), Y, W, X);
      release(t + 1);
    }
    if (t + 2 <= tl) {
      m.step(pfirst + dir * (t + 2), W, X, Y);
      release(t + 2);
    }
  }
  if (!m.ok && fault != nullptr) atomicExch(fault, 1);
}

template <typename T, bool ISO, int RC, int NWC, int NS>
static cudaError_t rr_rb_t(const Dims& fd, const Dims& cd, const double h[3], const void* phi, const void* fs,
                           void* fsc, double factor, int* fault, cudaStream_t s) {
  using Gm = RrbGeom<T, RC, NWC, NS>;
  auto kern = k_resid_restrict_rb<T, ISO, RC, NWC, NS>;
  static int blocks_per_sm = 0;
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, Gm::NTH, Gm::SMEM);
    if (e != cudaSuccess) return e;
    blocks_per_sm = std::max(1, blocks_per_sm);
  }
  const int dt = sizeof(T) == 4 ? DT_F32 : DT_BF16;
  CUtensorMap mP, mF;
  if (!encode_level_map(&mP, dt, phi, fd, Gm::WP, Gm::HP) || !encode_level_map(&mF, dt, fs, fd, Gm::WP, Gm::HF))
    return cudaErrorInvalidValue;
  const int gx = (cd.nx - 1) / Gm::TXC + 1, gy = (cd.ny - 1) / Gm::TYC + 1;
  const int nk = cd.nz - 1;
  const int slots = sm_count() * blocks_per_sm;
  const int nchunk = std::max(1, std::min(nk, slots / (gx * gy)));
  const int kc = (nk + nchunk - 1) / nchunk;
  const dim3 grid(gx, gy, (nk + kc - 1) / kc);
  const Coef<float> cf = make_coef<float>(fd, h, 2);
  kern<<<grid, Gm::NTH, Gm::SMEM, s>>>(mP, mF, fd, cd, cf, (float*)fsc, (float)(factor / 64.0), kc, fault);
  return cudaGetLastError();
}

template <typename TF, typename TC, int G, bool ISO>
static cudaError_t rr_t(const Dims& fd, const Dims& cd, const double h[3], int order, const void* phi,
                        const void* fs, void* fsc, double factor, int* fault, cudaStream_t s) {
  using C = typename St<TF>::C;
  constexpr int TXC = 32, TYC = sizeof(TF) == 8 ? 4 : 8;
  using Gm = RRGeom<TF, G, TXC, TYC>;
  const int smem = Gm::NS * (Gm::PB + Gm::FB) + align_up(Gm::DW * Gm::DH * (int)sizeof(C), 128) + Gm::NS * 8;
  auto kern = k_resid_restrict<TF, TC, G, ISO, TXC, TYC>;
  static int blocks_per_sm = 0;
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    blocks_per_sm = std::max(1, blocks_per_sm);
  }
  const int dt = sizeof(TF) == 8 ? DT_F64 : sizeof(TF) == 4 ? DT_F32 : DT_BF16;
  CUtensorMap mP, mF;
  if (!encode_level_map(&mP, dt, phi, fd, Gm::WP, Gm::HP) || !encode_level_map(&mF, dt, fs, fd, Gm::WP, Gm::HF))
    return cudaErrorInvalidValue;
  // coarse tiles cover nodes I in [bx * TXC, bx * TXC + TXC); interior nodes are 1 .. nc-1
  const int gx = (cd.nx - 1) / TXC + 1, gy = (cd.ny - 1) / TYC + 1;
  const int nk = cd.nz - 1;
  const int slots = sm_count() * blocks_per_sm;
  const int nchunk = std::max(1, std::min(nk, slots / (gx * gy)));
  const int kc = (nk + nchunk - 1) / nchunk;
  const dim3 grid(gx, gy, (nk + kc - 1) / kc);
  Coef<C> cf = make_coef<C>(fd, h, order);
  kern<<<grid, NT, smem, s>>>(mP, mF, fd, cd, cf, (TC*)fsc, (C)(factor / 64.0), kc, fault);
  return cudaGetLastError();
}

// Tile variants of k_resid_restrict_rb (coarse rows per warp x warps per block,
// 32 coarse columns, 5-stage ring): 1 = 4 x 4, 2 = 2 x 4, 3 = 3 x 4.  Every
// variant gives the same coarse right-hand side bit for bit.  Default 3 (12
// warps per SM; measured at 256^3 against 1 and 2, FP32 and BF16).
int rr_default_tile(int) { return 3; }

template <typename T, bool ISO>
static cudaError_t rr_rb_tile(const Dims& fd, const Dims& cd, const double h[3], const void* phi, const void* fs,
                              void* fsc, double factor, int* fault, int tile, cudaStream_t s) {
  switch (tile) {
    case 1: return rr_rb_t<T, ISO, 4, 4, 5>(fd, cd, h, phi, fs, fsc, factor, fault, s);
    case 2: return rr_rb_t<T, ISO, 2, 4, 5>(fd, cd, h, phi, fs, fsc, factor, fault, s);
    case 3: return rr_rb_t<T, ISO, 3, 4, 5>(fd, cd, h, phi, fs, fsc, factor, fault, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename TF, typename TC>
static cudaError_t rr_dispatch(const Dims& fd, const Dims& cd, int order, const double h[3], const void* phi,
                               const void* fs, void* fsc, double factor, int* fault, int tile, cudaStream_t s) {
  const bool iso = h[0] == h[1] && h[1] == h[2];
  if constexpr (!std::is_same<TF, double>::value && std::is_same<TC, float>::value) {
    if (order == 2) {
      if (tile == 0) tile = rr_default_tile(sizeof(TF) == 4 ? DT_F32 : DT_BF16);
      return iso ? rr_rb_tile<TF, true>(fd, cd, h, phi, fs, fsc, factor, fault, tile, s)
                 : rr_rb_tile<TF, false>(fd, cd, h, phi, fs, fsc, factor, fault, tile, s);
    }
  }
  if (order == 2)
    return iso ? rr_t<TF, TC, 1, true>(fd, cd, h, order, phi, fs, fsc, factor, fault, s)
               : rr_t<TF, TC, 1, false>(fd, cd, h, order, phi, fs, fsc, factor, fault, s);
  return iso ? rr_t<TF, TC, 2, true>(fd, cd, h, order, phi, fs, fsc, factor, fault, s)
             : rr_t<TF, TC, 2, false>(fd, cd, h, order, phi, fs, fsc, factor, fault, s);
}

cudaError_t launch_resid_restrict(const Dims& fine, const Dims& coarse, int order, const double h[3], int dt_f,
                                  const void* phi, const void* fs, int dt_c, void* fs_c,
                                  double factor, int* fault, cudaStream_t s, int tile) {
  if (tile < 0 || tile > kRrTiles) return cudaErrorInvalidValue;
  if (dt_f == DT_F64 && dt_c == DT_F64) return rr_dispatch<double, double>(fine, coarse, order, h, phi, fs, fs_c, factor, fault, tile, s);
  if (dt_f == DT_F32 && dt_c == DT_F32) return rr_dispatch<float, float>(fine, coarse, order, h, phi, fs, fs_c, factor, fault, tile, s);
  if (dt_f == DT_BF16 && dt_c == DT_F32) return rr_dispatch<__nv_bfloat16, float>(fine, coarse, order, h, phi, fs, fs_c, factor, fault, tile, s);
  return cudaErrorNotSupported;
}

// ================================================================== colour-restricted norm
// After an omega = 1 sweep the last colour's nodes have delta = 0 exactly; only
// the other colours' residuals are evaluated (one thread per such node and row
// position, as in the colour passes).  FP64 only (convergence checks).
template <int G, bool ISO>
__global__ void __launch_bounds__(256)
    k_delta_colours(Dims d, Coef<double> cf, const double* __restrict__ phi,
                    const double* __restrict__ fs, double* __restrict__ partials) {
  constexpr int NCOL = G == 1 ? 2 : 3;
  const int t = blockIdx.x * 32 + threadIdx.x;
  const int jn = blockIdx.y * 8 + threadIdx.y + 1;
  const int zc = (d.nk() + gridDim.z - 1) / gridDim.z;
  const int kn0 = blockIdx.z * zc + 1;
  const int kn1 = min(kn0 + zc, d.nk() + 1);
  const long long sy = d.sy(), sz = d.sz();
  double s2 = 0.0;
  if (jn <= d.nj()) {
    for (int kn = kn0; kn < kn1; kn++) {
#pragma unroll
      for (int colour = 0; colour < NCOL - 1; colour++) {
        const int r0 = ((colour - jn - kn - 1) % NCOL + NCOL) % NCOL;
        const int in = 1 + r0 + NCOL * t;
        if (in > d.ni()) continue;
        const long long p = d.at(in + G - 1, jn + G - 1, kn + G - 1);
        double ax = phi[p + 1] + phi[p - 1];
        double ay = phi[p + sy] + phi[p - sy];
        double az = phi[p + sz] + phi[p - sz];
        double v;
        if (ISO) v = fma((ax + ay) + az, cf.c1[0], fs[p]);
        else v = fma(ax, cf.c1[0], fma(ay, cf.c1[1], fma(az, cf.c1[2], fs[p])));
        if (G == 2) {
          const double bx = phi[p + 2] + phi[p - 2];
          const double by = phi[p + 2 * sy] + phi[p - 2 * sy];
          const double bz = phi[p + 2 * sz] + phi[p - 2 * sz];
          if (ISO) v = fma((bx + by) + bz, cf.c2[0], v);
          else v = fma(bx, cf.c2[0], fma(by, cf.c2[1], fma(bz, cf.c2[2], v)));
        }
        const double dl = v - phi[p];
        s2 = fma(dl, dl, s2);
      }
    }
  }
  // block sum -> partials[2 b], partials[2 b + 1] = 0
  __shared__ double sh[8];
  const int tid = threadIdx.x + 32 * threadIdx.y;
  s2 = warp_sum(s2);
  if ((tid & 31) == 0) sh[tid >> 5] = s2;
  __syncthreads();
  if (tid < 32) {
    double a = tid < 8 ? sh[tid] : 0.0;
    a = warp_sum(a);
    if (tid == 0) {
      const int b = block_linear_id();
      partials[2 * b] = a;
      partials[2 * b + 1] = 0.0;
    }
  }
}

// FP64 7-point on equal spacings: the red residuals along (j, k) diagonals,
// with the pair sum (N + U) of one node carried as the (S + D) of the next, in
// the order of the diagonal colour pass (5 + 1 FP64 instructions per node).
// Layout of the walks as in k_sweep_diag (x pair per thread, dl nodes per walk).
static dim3 diag_grid(const Dims& d) {
  const int dl = diag_walk_len(d.nk());
  const int pairs = (d.ni() + 1) / 2;
  return dim3((pairs + 31) / 32, (d.nj() + dl - 1 + 7) / 8, (d.nk() + dl - 1) / dl);
}

__global__ void __launch_bounds__(256)
    k_delta_red_diag(Dims d, double c1, const double* __restrict__ phi, const double* __restrict__ fs, int dl,
                     double* __restrict__ partials) {
  const int t = blockIdx.x * 32 + threadIdx.x;
  const int jn0 = blockIdx.y * 8 + threadIdx.y + 2 - dl;
  const int kn0 = blockIdx.z * dl + 1;
  const int ni = d.ni(), nj = d.nj(), nk = d.nk();
  const int u0 = jn0 < 1 ? 1 - jn0 : 0;
  const int u1 = min(dl, min(nj - jn0 + 1, nk - kn0 + 1));
  const int in = 1 + 2 * t + ((1 + jn0 + kn0) & 1);   // the red member of the pair
  double s2 = 0.0;
  if (u0 < u1 && in <= ni) {
    const long long sy = d.sy(), sz = d.sz(), step = sy + sz;
    long long c = d.at(in, jn0 + u0, kn0 + u0);
    double qprev = phi[c - sy] + phi[c - sz];
    // raw operands one node ahead, summed one step later (the last step reloads its own node)
    double e = phi[c + 1], w = phi[c - 1], nn = phi[c + sy], up = phi[c + sz], f = fs[c], x = phi[c];
    for (int u = u0; u < u1; u++) {
      const long long cn = u + 1 < u1 ? c + step : c;
      const double e2 = phi[cn + 1], w2 = phi[cn - 1], n2 = phi[cn + sy], u2 = phi[cn + sz], f2 = fs[cn], x2 = phi[cn];
      const double q = nn + up;
      const double dl_ = fma(((e + w) + qprev) + q, c1, f) - x;
      s2 = fma(dl_, dl_, s2);
      qprev = q;
      c += step;
      e = e2;
      w = w2;
      nn = n2;
      up = u2;
      f = f2;
      x = x2;
    }
  }
  __shared__ double sh[8];
  const int tid = threadIdx.x + 32 * threadIdx.y;
  s2 = warp_sum(s2);
  if ((tid & 31) == 0) sh[tid >> 5] = s2;
  __syncthreads();
  if (tid < 32) {
    double a = tid < 8 ? sh[tid] : 0.0;
    a = warp_sum(a);
    if (tid == 0) {
      const int b = block_linear_id();
      partials[2 * b] = a;
      partials[2 * b + 1] = 0.0;
    }
  }
}

static dim3 delta_colours_grid(const Dims& d, int order) {
  const int ncol = order == 2 ? 2 : 3;
  const int per_row = (d.ni() + ncol - 1) / ncol;
  const int gx = (per_row + 31) / 32, gy = (d.nj() + 7) / 8;
  const long long target = 8LL * sm_count();
  const int zc = (int)std::max(1LL, std::min(16LL, (long long)gx * gy * d.nk() / target));
  return dim3(gx, gy, (d.nk() + zc - 1) / zc);
}

int delta_colours_partials(const Dims& d, int order) {
  const dim3 g = delta_colours_grid(d, order), gd = diag_grid(d);
  return (int)std::max(g.x * g.y * g.z, order == 2 ? gd.x * gd.y * gd.z : (unsigned)delta_diag13_blocks(d));
}

cudaError_t launch_delta_colours(const Dims& d, int order, const double h[3], const double* phi,
                                 const double* fs, double* partials, int* nblocks, cudaStream_t s) {
  Coef<double> cf = make_coef<double>(d, h, order);
  const bool iso = h[0] == h[1] && h[1] == h[2];
  const dim3 blk(32, 8);
  if (order == 2 && iso) {
    const dim3 gd = diag_grid(d);
    if (nblocks) *nblocks = (int)(gd.x * gd.y * gd.z);
    k_delta_red_diag<<<gd, blk, 0, s>>>(d, cf.c1[0], phi, fs, diag_walk_len(d.nk()), partials);
    return cudaGetLastError();
  }
  if (order == 4 && iso) return launch_delta_diag13(d, h, 0, phi, fs, DT_F64, nullptr, nullptr, partials, nblocks, s);
  const dim3 grid = delta_colours_grid(d, order);
  if (nblocks) *nblocks = (int)(grid.x * grid.y * grid.z);
  if (order == 2) {
    if (iso) k_delta_colours<1, true><<<grid, blk, 0, s>>>(d, cf, phi, fs, partials);
    else k_delta_colours<1, false><<<grid, blk, 0, s>>>(d, cf, phi, fs, partials);
  } else {
    if (iso) k_delta_colours<2, true><<<grid, blk, 0, s>>>(d, cf, phi, fs, partials);
    else k_delta_colours<2, false><<<grid, blk, 0, s>>>(d, cf, phi, fs, partials);
  }
  return cudaGetLastError();
}

}  // namespace ps
