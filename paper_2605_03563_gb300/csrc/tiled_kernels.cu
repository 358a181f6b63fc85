// TMA-staged z-marching tile kernels of the GB300 Poisson library.
//
// Both kernels walk a z-chunk of planes per thread block.  A ring of NS plane
// buffers in shared memory is filled by TMA boxes (cp.async.bulk.tensor, one
// mbarrier per stage) several planes ahead of the plane being computed, so the
// HBM stream never waits on the arithmetic.  Every array they read is a
// library-layout level array (rows padded to 32 elements).
//
// k_rb_sweep: one whole red-black Gauss-Seidel sweep of the 7-point operator
//   (Sec. 2.1.1, red = (i+j+k) even first), out of place.  Red updates of a
//   plane are computed on the tile plus a one-node halo into a shared ring of
//   three planes; black updates read only that ring.  Halo red values equal the
//   neighbouring tile's (same operands, same arithmetic), so the result is the
//   sequential red-then-black sweep bit for bit, while HBM traffic is one read
//   of phi and fs and one write of phi per sweep instead of per colour.
//
// k_resid_restrict: the fine residual delta = phi_GS - phi of each plane is
//   computed into shared memory on the tile's (2T+1)^2 footprint and folded at
//   once into the full-weighting sums of the coarse nodes (Sec. 2.1.3); the
//   fine residual never reaches HBM.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

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

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

static constexpr int NT = 256;   // threads per block of both tile kernels

// x halo of a staged box: at least 2 nodes and a whole 16-byte TMA granule
template <typename T>
__host__ __device__ constexpr int xhalo() {
  return sizeof(T) >= 8 ? 2 : (int)(16 / sizeof(T));
}

// ================================================================== red-black sweep
// Block = NW = TY + 2 warps over a 64 x TY tile.  Warp w owns ring row w, i.e.
// grid row y = y0 - 1 + w (w = 0 and w = TY + 1 are halo rows that only
// compute red values); lane l owns the x pair (x0 + 2l, x0 + 2l + 1), of which
// exactly one node is red on every plane.  Because x0 is even, the red column
// of a row alternates with the plane and is the same for all lanes of a warp,
// so the warp never diverges on colour.  The red node of a lane on plane z and
// on plane z +- 2 is the same column, so each lane keeps in registers the red
// values of planes k-1, k, k+1 (the black update's z neighbours and the red
// half of the output pair) and the old potential of its red column one plane
// up (the next-but-one red update's lower z neighbour).  Warp 0 also computes
// the red values of the two halo columns x0 - 1 and x0 + 64 (one of them is red
// in each row), which the edge lanes' black updates read.
template <typename T, int TY, int NS>
struct SweepGeom {
  static constexpr int TX = 64;
  static constexpr int NW = TY + 2;                // warps: ring rows y0-1 .. y0+TY
  static constexpr int NTH = 32 * NW;
  static constexpr int XH = xhalo<T>();
  static constexpr int WP = TX + 2 * XH;           // staged row width (phi and fs)
  static constexpr int HP = TY + 4;                // phi rows: y0-2 .. y0+TY+1
  static constexpr int HF = TY + 2;                // fs rows:  y0-1 .. y0+TY
  static constexpr int RW = TX + 2, RH = TY + 2;   // red ring: x0-1..x0+TX, y0-1..y0+TY
  static constexpr int PBYTES = WP * HP * (int)sizeof(T);
  static constexpr int FBYTES = WP * HF * (int)sizeof(T);
  static constexpr int PB = align_up(PBYTES, 128), FB = align_up(FBYTES, 128);
  static constexpr int RB = align_up(RW * RH * (int)sizeof(T), 128);
  static constexpr int SMEM = NS * (PB + FB) + 3 * RB + NS * 8;
};

template <typename T, bool ISO, int TY, int NS>
__global__ void __launch_bounds__(32 * (TY + 2))
    k_rb_sweep(const __grid_constant__ CUtensorMap mP, const __grid_constant__ CUtensorMap mF, Dims d,
               Coef<typename St<T>::C> cf, T* __restrict__ out, int zc, const DevState* __restrict__ st,
               int* __restrict__ fault) {
  using C = typename St<T>::C;
  using S = St<T>;
  using Gm = SweepGeom<T, TY, NS>;
  constexpr int TX = Gm::TX, NW = Gm::NW, XH = Gm::XH, WP = Gm::WP, RW = Gm::RW;
  constexpr int PBE = Gm::PB / (int)sizeof(T), FBE = Gm::FB / (int)sizeof(T), RBE = Gm::RB / (int)sizeof(T);
  extern __shared__ __align__(128) unsigned char smem[];
  T* Pst = reinterpret_cast<T*>(smem);
  T* Fst = reinterpret_cast<T*>(smem + NS * Gm::PB);
  T* Rr = reinterpret_cast<T*>(smem + NS * (Gm::PB + Gm::FB));
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + NS * (Gm::PB + Gm::FB) + 3 * Gm::RB);

  if (st != nullptr && st->done) return;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int nx = d.nx, ny = d.ny, nz = d.nz;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = 1 + blockIdx.z * zc;
  const int z1 = min(z0 + zc, nz);     // output planes [z0, z1)
  const int zl = z0 - 2, zh = z1 + 1;  // staged planes [zl, zh]; plane z sits in stage (z - zl) % NS
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
  // planes are waited for in order; (wq, wph) = stage and phase of the next one
  bool ok = true;
  int wq = 0;
  unsigned wph = 0;
  auto wait_next = [&]() {
    mbar_wait(&bar[wq], wph, ok);
    if (++wq == NS) { wq = 0; wph ^= 1u; }
  };
  auto nxt = [](int q) { return q + 1 == NS ? 0 : q + 1; };

  const int y = y0 - 1 + w;                        // this warp's grid row
  const bool row_out = w >= 1 && w <= TY && y >= 1 && y < ny;
  const bool row_bnd = y <= 0 || y >= ny;
  const int xa = x0 + 2 * l;
  // boundary or outside in x, for the pair's even / odd column
  const bool bnd_e = row_bnd || xa <= 0 || xa >= nx;
  const bool bnd_o = row_bnd || xa + 1 >= nx;
  const bool st_pair = row_out && xa >= 1 && xa + 1 < nx;
  const bool st_a = row_out && xa >= 1 && xa < nx, st_b = row_out && xa + 1 < nx;
  const int pbase = (w + 1) * WP + XH + 2 * l;     // P index of (xa, y)
  const int fbase = w * WP + XH + 2 * l;           // F index of (xa, y)
  const int rbase = w * RW + 1 + 2 * l;            // R index of (xa, y)

  // red value at column xa + par of this warp's row on plane z (stage qz, plane z+1 in
  // stage qp), zm = old phi one plane down; returns the value as stored
  auto red_at = [&](int par, bool zb, int qz, int qp, C zm) -> C {
    const T* P = Pst + qz * PBE + pbase + par;
    C v;
    if (zb || (par ? bnd_o : bnd_e)) {
      v = S::ld(P);
    } else {
      const C ax = S::ld(P + 1) + S::ld(P - 1);
      const C ay = S::ld(P + WP) + S::ld(P - WP);
      const C az = S::ld(Pst + qp * PBE + pbase + par) + zm;
      const C f = S::ld(Fst + qz * FBE + fbase + par);
      if (ISO) v = fma((ax + ay) + az, cf.c1[0], f);
      else v = fma(ax, cf.c1[0], fma(ay, cf.c1[1], fma(az, cf.c1[2], f)));
    }
    return stored<T>(v);
  };
  // warp 0: red value of the halo column of ring row l (l < NW) on plane z
  auto halo_red = [&](int z, int qm, int qz, int qp, T* R) {
    if (w != 0 || l >= NW) return;
    const int yy = y0 - 1 + l;
    const int hc = ((yy + z) & 1) ? x0 - 1 : x0 + TX;
    const T* P = Pst + qz * PBE;
    const int pc = (l + 1) * WP + XH + (hc - x0);
    C v;
    if (yy <= 0 || yy >= ny || z <= 0 || z >= nz || hc <= 0 || hc >= nx) {
      v = S::ld(P + pc);
    } else {
      const C ax = S::ld(P + pc + 1) + S::ld(P + pc - 1);
      const C ay = S::ld(P + pc + WP) + S::ld(P + pc - WP);
      const C az = S::ld(Pst + qp * PBE + pc) + S::ld(Pst + qm * PBE + pc);
      const C f = S::ld(Fst + qz * FBE + l * WP + XH + (hc - x0));
      if (ISO) v = fma((ax + ay) + az, cf.c1[0], f);
      else v = fma(ax, cf.c1[0], fma(ay, cf.c1[1], fma(az, cf.c1[2], f)));
    }
    S::st(R + l * RW + 1 + (hc - x0), v);
  };

  if (tid == 0)
    for (int q = 0; q < NS; q++) issue(zl + q, q);
  // prologue: red values of planes z0-1 (stages 0,1,2 = planes z0-2, z0-1, z0) and z0
  wait_next();
  wait_next();
  wait_next();
  C rm2, rm1, ph0, ph1;   // red(k-1), red(k); old phi one plane above the red column of planes k+1, k+2
  {
    const int z = z0 - 1, par = (y + z) & 1;
    const C zm = S::ld(Pst + 0 * PBE + pbase + par);
    rm2 = red_at(par, z <= 0, 1, 2, zm);
    S::st(Rr + 0 * RBE + rbase + par, rm2);
    ph0 = S::ld(Pst + 2 * PBE + pbase + par);   // phi(z0) at the red column of planes z0-1, z0+1
    halo_red(z, 0, 1, 2, Rr + 0 * RBE);
  }
  wait_next();   // plane z0 + 1 in stage 3
  {
    const int z = z0, par = (y + z) & 1;
    const C zm = S::ld(Pst + 1 * PBE + pbase + par);
    rm1 = red_at(par, false, 2, 3, zm);
    S::st(Rr + 1 * RBE + rbase + par, rm1);
    ph1 = S::ld(Pst + 3 * PBE + pbase + par);   // phi(z0+1) at the red column of planes z0, z0+2
    halo_red(z, 1, 2, 3, Rr + 1 * RBE);
  }
  __syncthreads();
  if (tid == 0) {
    fence_proxy_async();
    issue(zl + NS, 0);
  }
  // rotating stages of planes k, k+1, k+2 and ring slots of planes k, k+1
  int qk = 2, qk1 = 3, qk2 = 4 % NS, iq = 1;
  T* Rk = Rr + 1 * RBE;
  T* Rk1 = Rr + 2 * RBE;
  T* Rk2 = Rr + 0 * RBE;
  T* o = out + ((long long)z0 * d.ey + y) * d.px + xa;
  const long long osz = d.sz();
  for (int k = z0; k < z1; k++) {
    wait_next();   // plane k + 2
    const int zr = k + 1, par = (y + zr) & 1;
    const C rp = red_at(par, zr >= nz, qk1, qk2, ph0);
    S::st(Rk1 + rbase + par, rp);
    ph0 = ph1;
    ph1 = S::ld(Pst + qk2 * PBE + pbase + par);
    halo_red(zr, qk, qk1, qk2, Rk1);
    __syncthreads();
    if (tid == 0) {
      fence_proxy_async();
      issue(k - 1 + NS, iq);   // stage of plane k-1
    }
    if (row_out) {
      // black(k) at column xa + par (black on plane k), red(k) at the other column
      const T* Rb = Rk + rbase + par;
      const C ax = S::ld(Rb + 1) + S::ld(Rb - 1);
      const C ay = S::ld(Rb + RW) + S::ld(Rb - RW);
      const C az = rp + rm2;
      const C f = S::ld(Fst + qk * FBE + fbase + par);
      C vb;
      if (ISO) vb = fma((ax + ay) + az, cf.c1[0], f);
      else vb = fma(ax, cf.c1[0], fma(ay, cf.c1[1], fma(az, cf.c1[2], f)));
      const C v0 = par ? rm1 : vb, v1 = par ? vb : rm1;
      if (st_pair) {
        St2<T>::st(o, v0, v1);
      } else {
        if (st_a) S::st(o, v0);
        if (st_b) S::st(o + 1, v1);
      }
    }
    o += osz;
    rm2 = rm1;
    rm1 = rp;
    T* t = Rk;
    Rk = Rk1;
    Rk1 = Rk2;
    Rk2 = t;
    iq = qk;
    qk = qk1;
    qk1 = qk2;
    qk2 = nxt(qk2);
  }
  if (!ok && fault != nullptr) atomicExch(fault, 1);
}

template <typename T, bool ISO>
static cudaError_t rb_sweep_t(const Dims& d, const double h[3], const void* pin, void* pout,
                              const void* fs, const DevState* st, int* fault, cudaStream_t s) {
  using C = typename St<T>::C;
  // 6 planes in the ring (3 in flight) keep 3 blocks of 512 threads per SM for FP32;
  // deeper rings measured slower (fewer resident blocks)
  constexpr int TY = 14, NS = 6;
  using Gm = SweepGeom<T, TY, NS>;
  auto kern = k_rb_sweep<T, ISO, TY, NS>;
  static int blocks_per_sm = 0;
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, Gm::NTH, Gm::SMEM);
    if (e != cudaSuccess) return e;
    blocks_per_sm = std::max(1, blocks_per_sm);
  }
  const int dt = sizeof(T) == 8 ? DT_F64 : sizeof(T) == 4 ? DT_F32 : DT_BF16;
  CUtensorMap mP, mF;
  if (!encode_level_map(&mP, dt, pin, d, Gm::WP, Gm::HP) || !encode_level_map(&mF, dt, fs, d, Gm::WP, Gm::HF))
    return cudaErrorInvalidValue;
  const int gx = (d.nx - 1) / Gm::TX + 1, gy = (d.ny - 1) / TY + 1;
  const int nk = d.nz - 1;
  // one wave: as many z-chunks per tile column as keep every block resident
  const int slots = sm_count() * blocks_per_sm;
  const int nchunk = std::max(1, std::min(nk, slots / (gx * gy)));
  const int zc = (nk + nchunk - 1) / nchunk;
  const dim3 grid(gx, gy, (nk + zc - 1) / zc);
  Coef<C> cf = make_coef<C>(d, h, 2);
  kern<<<grid, Gm::NTH, Gm::SMEM, s>>>(mP, mF, d, cf, (T*)pout, zc, st, fault);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t rb_sweep_dispatch(const Dims& d, const double h[3], const void* pin, void* pout,
                                     const void* fs, const DevState* st, int* fault, cudaStream_t s) {
  if (h[0] == h[1] && h[1] == h[2]) return rb_sweep_t<T, true>(d, h, pin, pout, fs, st, fault, s);
  return rb_sweep_t<T, false>(d, h, pin, pout, fs, st, fault, s);
}

// FP64 levels keep the colour passes (their sweeps are bound by the FP64 pipe),
// so the fused sweep is built for the FP32 and BF16 inner levels only.
cudaError_t launch_rb_sweep(const Dims& d, int order, const double h[3], int dt, const void* phi_in,
                            void* phi_out, const void* fs, const DevState* st, int* fault,
                            cudaStream_t s) {
  if (order != 2 || d.g != 1 || dt == DT_F64) return cudaErrorNotSupported;
  if (dt == DT_F32) return rb_sweep_dispatch<float>(d, h, phi_in, phi_out, fs, st, fault, s);
  return rb_sweep_dispatch<__nv_bfloat16>(d, h, phi_in, phi_out, fs, st, fault, s);
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
    if (tid == 0) {
      fence_proxy_async();
      issue(pc - G + NS);   // stage of phi plane pc - G
    }
    qc = wrap(qc + 1);
  }
  wait_upto(pz_hi);
  if (!ok && fault != nullptr) atomicExch(fault, 1);
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

template <typename TF, typename TC>
static cudaError_t rr_dispatch(const Dims& fd, const Dims& cd, int order, const double h[3], const void* phi,
                               const void* fs, void* fsc, double factor, int* fault, cudaStream_t s) {
  const bool iso = h[0] == h[1] && h[1] == h[2];
  if (order == 2)
    return iso ? rr_t<TF, TC, 1, true>(fd, cd, h, order, phi, fs, fsc, factor, fault, s)
               : rr_t<TF, TC, 1, false>(fd, cd, h, order, phi, fs, fsc, factor, fault, s);
  return iso ? rr_t<TF, TC, 2, true>(fd, cd, h, order, phi, fs, fsc, factor, fault, s)
             : rr_t<TF, TC, 2, false>(fd, cd, h, order, phi, fs, fsc, factor, fault, s);
}

cudaError_t launch_resid_restrict(const Dims& fine, const Dims& coarse, int order, const double h[3], int dt_f,
                                  const void* phi, const void* fs, int dt_c, void* fs_c,
                                  double factor, int* fault, cudaStream_t s) {
  if (dt_f == DT_F64 && dt_c == DT_F64) return rr_dispatch<double, double>(fine, coarse, order, h, phi, fs, fs_c, factor, fault, s);
  if (dt_f == DT_F32 && dt_c == DT_F32) return rr_dispatch<float, float>(fine, coarse, order, h, phi, fs, fs_c, factor, fault, s);
  if (dt_f == DT_BF16 && dt_c == DT_F32) return rr_dispatch<__nv_bfloat16, float>(fine, coarse, order, h, phi, fs, fs_c, factor, fault, s);
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

static dim3 delta_colours_grid(const Dims& d, int order) {
  const int ncol = order == 2 ? 2 : 3;
  const int per_row = (d.ni() + ncol - 1) / ncol;
  const int gx = (per_row + 31) / 32, gy = (d.nj() + 7) / 8;
  const long long target = 8LL * sm_count();
  const int zc = (int)std::max(1LL, std::min(16LL, (long long)gx * gy * d.nk() / target));
  return dim3(gx, gy, (d.nk() + zc - 1) / zc);
}

int delta_colours_partials(const Dims& d, int order) {
  const dim3 g = delta_colours_grid(d, order);
  return (int)(g.x * g.y * g.z);
}

cudaError_t launch_delta_colours(const Dims& d, int order, const double h[3], const double* phi,
                                 const double* fs, double* partials, int* nblocks, cudaStream_t s) {
  const dim3 grid = delta_colours_grid(d, order);
  if (nblocks) *nblocks = (int)(grid.x * grid.y * grid.z);
  Coef<double> cf = make_coef<double>(d, h, order);
  const bool iso = h[0] == h[1] && h[1] == h[2];
  const dim3 blk(32, 8);
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
