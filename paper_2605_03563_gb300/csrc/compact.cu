// Compact radius-one stencils, SPAI smoothing and Galerkin coarse operators
// (Sec. 2.1.3): FP64 passes, and the FP32 passes of the refinement's inner
// cycles.
//
// Compact schemes L_h u = R_h f of order 2, 4, 6 (isotropic spacing; weights
// from Taylor matching, as the paper cites compact schemes without printing
// them):
//   order 2: L = (-6, 1, 0, 0)/h^2,          R f = f
//   order 4: L = (-24, 2, 1, 0)/(6 h^2),     R f = f/2 + (1/12) sum_faces f
//   order 6: L = (-128, 14, 3, 1)/(30 h^2),  R f = (67/120) f + (1/18) sum_faces f
//            + (1/90) sum_edges f - (1/240) sum_{+-2 e_a} f
// (weights per offset class centre / faces / edges / corners).  The +-2
// offsets of the order-6 right-hand side reach one layer past the node array
// at the first interior layer; there f is the cubic extrapolation
// 4 f_0 - 6 f_1 + 4 f_2 - f_3 along that axis.
//
// The 27-point kernels march z and form per plane the in-plane sums C
// (centre), F (4 in-plane faces), E (4 in-plane diagonals), so that
//   (A u)(z) = w0 C(z) + w1 (F(z) + C(z-1) + C(z+1)) + w2 (E(z) + F(z-1) + F(z+1))
//            + w3 (E(z-1) + E(z+1))
//            = P(z) + Q(z-1) + Q(z+1),  P = w0 C + w1 F + w2 E,  Q = w1 C + w2 F + w3 E;
// a thread owns several rows of a column, so the pair sums u(x-1) + u(x+1)
// serve the rows above and below as well (12.5 FP64 operations per node for
// a residual instead of 27 multiply-adds).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "cart_kernels.cuh"
#include "compact.cuh"
#include "stencil.cuh"
#include "tma.cuh"

namespace ps {

static constexpr int CBX = 32, CBY = 8, CZC = 16;

W27 compact_lhs(int order, double h) {
  const double ih2 = 1.0 / (h * h);
  W27 a{};
  if (order == 2) {
    a = W27{{-6.0, 1.0, 0.0, 0.0}};
  } else if (order == 4) {
    a = W27{{-24.0 / 6.0, 2.0 / 6.0, 1.0 / 6.0, 0.0}};
  } else {
    a = W27{{-128.0 / 30.0, 14.0 / 30.0, 3.0 / 30.0, 1.0 / 30.0}};
  }
  for (double& v : a.w) v *= ih2;
  return a;
}

// R A P on a 9^3-node fine grid around one coarse delta: prolong the delta
// (trilinear: per axis 1, 1/2), apply A on the fine interior, restrict with
// full weighting (per axis 1/4, 1/2, 1/4) at the coarse neighbours.
W27 galerkin27(const W27& A) {
  const int N = 9;   // fine nodes 0..8, coarse delta at fine node 4 (coarse node 2)
  auto idx = [&](int i, int j, int k) { return (k * N + j) * N + i; };
  std::vector<double> pe(N * N * N, 0.0), ape(N * N * N, 0.0);
  auto wp = [](int d) { return d == 0 ? 1.0 : (std::abs(d) == 1 ? 0.5 : 0.0); };
  for (int k = 0; k < N; k++)
    for (int j = 0; j < N; j++)
      for (int i = 0; i < N; i++) pe[idx(i, j, k)] = wp(i - 4) * wp(j - 4) * wp(k - 4);
  for (int k = 1; k < N - 1; k++)
    for (int j = 1; j < N - 1; j++)
      for (int i = 1; i < N - 1; i++) {
        double s = 0.0;
        for (int dz = -1; dz <= 1; dz++)
          for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++)
              s += A.w[(dx != 0) + (dy != 0) + (dz != 0)] * pe[idx(i + dx, j + dy, k + dz)];
        ape[idx(i, j, k)] = s;
      }
  auto wr = [](int d) { return d == 0 ? 0.5 : 0.25; };
  double sum[4] = {0, 0, 0, 0};
  int cnt[4] = {0, 0, 0, 0};
  for (int Dz = -1; Dz <= 1; Dz++)
    for (int Dy = -1; Dy <= 1; Dy++)
      for (int Dx = -1; Dx <= 1; Dx++) {
        double s = 0.0;
        for (int ez = -1; ez <= 1; ez++)
          for (int ey = -1; ey <= 1; ey++)
            for (int ex = -1; ex <= 1; ex++)
              s += wr(ex) * wr(ey) * wr(ez) * ape[idx(4 + 2 * Dx + ex, 4 + 2 * Dy + ey, 4 + 2 * Dz + ez)];
        const int c = (Dx != 0) + (Dy != 0) + (Dz != 0);
        sum[c] += s;
        cnt[c]++;
      }
  W27 out;
  for (int c = 0; c < 4; c++) out.w[c] = sum[c] / cnt[c];
  return out;
}

// in-plane sums of plane k at (i, j): centre, 4 faces, 4 diagonals
template <typename C>
struct Plane {
  C c, f, e;
};

// the 3 x 3 neighbourhood of (i, j) on plane k (ZI: interior nodes read as 0)
template <typename C>
struct Raw9 {
  C c, xm, xp, ym, yp, mm, pm, mp, pp;
};

template <bool ZI, typename T, typename C = typename St<T>::C>
__device__ __forceinline__ Raw9<C> plane_load(const Dims& d, const T* __restrict__ u, int i, int j, int k) {
  const long long sy = d.sy();
  const long long p = d.at(i, j, k);
  auto ld = [&](long long q, int ii, int jj) -> C {
    if (ZI && ii >= 1 && ii <= d.ni() && jj >= 1 && jj <= d.nj() && k >= 1 && k <= d.nk()) return (C)0;
    return (C)u[q];
  };
  Raw9<C> v;
  v.c = ld(p, i, j);
  v.xm = ld(p - 1, i - 1, j);
  v.xp = ld(p + 1, i + 1, j);
  v.ym = ld(p - sy, i, j - 1);
  v.yp = ld(p + sy, i, j + 1);
  v.mm = ld(p - sy - 1, i - 1, j - 1);
  v.pm = ld(p - sy + 1, i + 1, j - 1);
  v.mp = ld(p + sy - 1, i - 1, j + 1);
  v.pp = ld(p + sy + 1, i + 1, j + 1);
  return v;
}

template <typename C>
__device__ __forceinline__ Plane<C> plane_of(const Raw9<C>& v) {
  Plane<C> s;
  s.c = v.c;
  s.f = (v.xm + v.xp) + (v.ym + v.yp);
  s.e = (v.mm + v.pm) + (v.mp + v.pp);
  return s;
}

// stencil weights in the arithmetic precision of the kernel (converted on the host)
template <typename C>
struct Wts {
  C w[4];
};

// Per-plane split of a 27-point class stencil w (centre, faces, edges,
// corners): with the in-plane sums (C, F, E) of planes z - 1, z, z + 1,
//   (A u)(z) = P(z) + Q(z - 1) + Q(z + 1),
//   P = w0 C + w1 F + w2 E,   Q = w1 C + w2 F + w3 E,
// so each plane's Q serves the nodes above and below it.  With nw = -s w
// (s = 1 for a residual, omega for a SPAI step) the pass value is
//   base - s P - s Q(z - 1) - s Q(z + 1) = base + nP + (nQ(z - 1) + nQ(z + 1)).
template <typename C>
__device__ __forceinline__ C plane_q(const C nw[4], const Plane<C>& p) {
  return fma(nw[1], p.c, fma(nw[2], p.f, nw[3] * p.e));
}
template <typename C>
__device__ __forceinline__ C plane_p_plus(const C nw[4], const Plane<C>& p, C base, C qm, C qp) {
  return fma(nw[0], p.c, fma(nw[1], p.f, fma(nw[2], p.e, base))) + (qm + qp);
}

// FP64 value stored as TR; FP32 stores round on the integer pipe (ties to
// even, the same value as the conversion instruction) instead of taking an
// FP64-pipe conversion.
template <typename TR>
__device__ __forceinline__ TR store_as(double v) {
  if constexpr (std::is_same<TR, float>::value) return f64_to_f32_pow2(v, 0);
  else return (TR)v;
}

// per-block {sum, 0} into partials[2 b], partials[2 b + 1] for blocks of NT threads
template <int NT>
__device__ __forceinline__ void block_partial_nt(double v, double* __restrict__ partials) {
  __shared__ double sh[NT / 32];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  v = warp_sum(v);
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    double a = tid < NT / 32 ? sh[tid] : 0.0;
    a = warp_sum(a);
    if (tid == 0) {
      const int bid = block_linear_id();
      partials[2 * bid] = a;
      partials[2 * bid + 1] = 0.0;
    }
  }
}

// per-block {v, 0} into p[2 b], p[2 b + 1] and {w, 0} into q[2 b], q[2 b + 1], blocks of NT threads
template <int NT>
__device__ __forceinline__ void block_partial2_nt(double v, double w, double* __restrict__ p,
                                                  double* __restrict__ q) {
  __shared__ double sh[2][NT / 32];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  v = warp_sum(v);
  w = warp_sum(w);
  if ((tid & 31) == 0) {
    sh[0][tid >> 5] = v;
    sh[1][tid >> 5] = w;
  }
  __syncthreads();
  if (tid < 32) {
    double a = tid < NT / 32 ? sh[0][tid] : 0.0;
    double c = tid < NT / 32 ? sh[1][tid] : 0.0;
    a = warp_sum(a);
    c = warp_sum(c);
    if (tid == 0) {
      const int bid = block_linear_id();
      p[2 * bid] = a;
      p[2 * bid + 1] = 0.0;
      q[2 * bid] = c;
      q[2 * bid + 1] = 0.0;
    }
  }
}

// FP64 passes (GB300's FP64 pipe bounds them, so they minimise FP64
// instructions): MODE 0: r = b - A u stored as TR (ZI: u's interior read as 0),
// per-block partials of r^2 if given; MODE 1: u -= omega M r.  A thread owns
// FRB consecutive rows of one column and marches z: per plane it loads the
// FRB + 2 rows x 3 columns around them, forms the pair sums u(x-1) + u(x+1)
// once per row and from them the in-plane sums (centre, faces, diagonals) of
// its rows, and applies the per-plane split P(z) + Q(z - 1) + Q(z + 1) of the
// stencil: 12.5 FP64 operations per node.  The loads of plane k + 2 are issued
// before the arithmetic of plane k.  Blocks of 32 x (CBY / FRB) threads cover
// the 32 x 8 tiles of c27_grid, so the partials count is c27_blocks(d).
// INIT (initial residual of a compact solve): also the reference residual
// b - A u0 of the boundary data alone (u0: u with its interior zeroed), whose
// partials go to partials + 2 nblocks; A u0 vanishes unless a node has a
// boundary node among its 26 neighbours, so only the first and last interior
// layers of each axis evaluate it (per node, with zero-interior loads), and
// elsewhere the reference residual is b.
static constexpr int FRB = 4;
template <int MODE, bool ZI, typename TR, bool NORM, bool INIT = false>
__global__ void __launch_bounds__(CBX*(CBY / FRB))
    k_c27_f64(Dims d, Wts<double> W, double om, const double* __restrict__ src, const double* __restrict__ b,
              TR* __restrict__ dst, double* __restrict__ partials, const DevState* __restrict__ st,
              int nblocks = 0) {
  if (st != nullptr && st->done) return;   // uniform
  const int i = blockIdx.x * CBX + threadIdx.x + 1;
  const int j0 = blockIdx.y * CBY + threadIdx.y * FRB + 1;   // rows j0 .. j0 + FRB - 1
  const int k0 = blockIdx.z * CZC + 1, k1 = min(k0 + CZC, d.nk() + 1);
  double s2 = 0.0, s0 = 0.0;
  if (i <= d.ni() && j0 <= d.nj()) {
    Wts<double> nw;
#pragma unroll
    for (int a = 0; a < 4; a++) nw.w[a] = MODE == 0 ? -W.w[a] : -om * W.w[a];
    const long long sz = d.sz();
    // rows j0 - 1 + s; rows past the ghost row nj + 1 are clamped to it: they
    // only feed rows that are not written
    long long roff[FRB + 2];
    bool rin[FRB + 2];
#pragma unroll
    for (int s = 0; s < FRB + 2; s++) {
      const int y = min(j0 - 1 + s, d.nj() + 1);
      roff[s] = (long long)y * d.sy() + i;
      rin[s] = y >= 1 && y <= d.nj();
    }
    const bool cin = i >= 1 && i <= d.ni(), lin = i - 1 >= 1, hin = i + 1 <= d.ni();
    // raw values of one plane: rows s = 0 .. FRB + 1, columns i - 1, i, i + 1
    auto load = [&](int k, double (&v)[FRB + 2][3]) {
      const double* p = src + (long long)k * sz;
      const bool kin = k >= 1 && k <= d.nk();
#pragma unroll
      for (int s = 0; s < FRB + 2; s++) {
        v[s][0] = (ZI && kin && rin[s] && lin) ? 0.0 : p[roff[s] - 1];
        v[s][1] = (ZI && kin && rin[s] && cin) ? 0.0 : p[roff[s]];
        v[s][2] = (ZI && kin && rin[s] && hin) ? 0.0 : p[roff[s] + 1];
      }
    };
    // in-plane sums of the thread's rows and their Q
    auto sums = [&](const double (&v)[FRB + 2][3], double (&C)[FRB], double (&F)[FRB], double (&E)[FRB],
                    double (&Q)[FRB]) {
      double a[FRB + 2];
#pragma unroll
      for (int s = 0; s < FRB + 2; s++) a[s] = v[s][0] + v[s][2];
#pragma unroll
      for (int q = 0; q < FRB; q++) {
        C[q] = v[q + 1][1];
        F[q] = a[q + 1] + (v[q][1] + v[q + 2][1]);
        E[q] = a[q] + a[q + 2];
        Q[q] = fma(nw.w[1], C[q], fma(nw.w[2], F[q], nw.w[3] * E[q]));
      }
    };
    double v[FRB + 2][3], vn[FRB + 2][3];
    double C[FRB], F[FRB], E[FRB], qm[FRB], qc[FRB];
    {
      double tC[FRB], tF[FRB], tE[FRB];
      load(k0 - 1, v);
      sums(v, tC, tF, tE, qm);
    }
    load(k0, v);
    sums(v, C, F, E, qc);
    load(k0 + 1, v);
    // b (MODE 0) or the residual being updated (MODE 1) of the thread's rows on
    // plane k, loaded one plane ahead like the stencil operands (the thread
    // writes only plane k of its own rows before it reads plane k + 1)
    auto load_b = [&](int k, double (&bb)[FRB]) {
      const long long base = (long long)k * sz;
#pragma unroll
      for (int q = 0; q < FRB; q++) {
        const long long o = base + roff[q + 1];
        bb[q] = j0 + q <= d.nj() ? (MODE == 0 ? b[o] : (double)dst[o]) : 0.0;
      }
    };
    double bc[FRB];
    load_b(k0, bc);
    for (int k = k0; k < k1; k++) {
      if (k + 2 <= k1) load(k + 2, vn);   // plane k1 <= nk + 1 exists
      double bn[FRB];
      load_b(k + 1 < k1 ? k + 1 : k, bn);
      double nC[FRB], nF[FRB], nE[FRB], qn[FRB];
      sums(v, nC, nF, nE, qn);
      const long long base = (long long)k * sz;
#pragma unroll
      for (int q = 0; q < FRB; q++) {
        if (j0 + q <= d.nj()) {
          const long long o = base + roff[q + 1];
          const double bv = bc[q];
          const double val = fma(nw.w[0], C[q], fma(nw.w[1], F[q], fma(nw.w[2], E[q], bv))) + (qm[q] + qn[q]);
          dst[o] = store_as<TR>(val);
          if (MODE == 0 && NORM) s2 = fma(val, val, s2);
          if constexpr (INIT) {
            // reference residual b - A u0 (u0: u with its interior zeroed); A u0
            // vanishes unless a boundary node is among the 26 neighbours
            const int j = j0 + q;
            double r0 = bv;
            if (i == 1 || i == d.ni() || j == 1 || j == d.nj() || k == 1 || k == d.nk())
              r0 = plane_p_plus(nw.w, plane_of(plane_load<true>(d, src, i, j, k)), bv,
                                plane_q(nw.w, plane_of(plane_load<true>(d, src, i, j, k - 1))),
                                plane_q(nw.w, plane_of(plane_load<true>(d, src, i, j, k + 1))));
            s0 = fma(r0, r0, s0);
          }
        }
        qm[q] = qc[q];
        qc[q] = qn[q];
        C[q] = nC[q];
        F[q] = nF[q];
        E[q] = nE[q];
        bc[q] = bn[q];
      }
#pragma unroll
      for (int s = 0; s < FRB + 2; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) v[s][c] = vn[s][c];
    }
  }
  if constexpr (INIT) block_partial2_nt<CBX*(CBY / FRB)>(s2, s0, partials, partials + 2 * nblocks);
  else if (MODE == 0 && NORM && partials != nullptr) block_partial_nt<CBX*(CBY / FRB)>(s2, partials);
}

template <typename C>
static Wts<C> wts(const W27& a) {
  return Wts<C>{{(C)a.w[0], (C)a.w[1], (C)a.w[2], (C)a.w[3]}};
}

static dim3 c27_grid(const Dims& d) {
  return dim3((d.ni() + CBX - 1) / CBX, (d.nj() + CBY - 1) / CBY, (d.nk() + CZC - 1) / CZC);
}

int c27_blocks(const Dims& d) {
  const dim3 g = c27_grid(d);
  return (int)(g.x * g.y * g.z);
}

cudaError_t launch_c27_resid(const Dims& d, const W27& A, const double* u, const double* b, double* r,
                             double* partials, const DevState* st, cudaStream_t s) {
  return launch_c27_resid_dt(d, A, u, b, DT_F64, r, partials, st, s);
}

cudaError_t launch_c27_resid_dt(const Dims& d, const W27& A, const double* u, const double* b, int dt_r, void* r,
                                double* partials, const DevState* st, cudaStream_t s) {
  if (d.g != 1) return cudaErrorInvalidValue;
  const dim3 g = c27_grid(d), b64(CBX, CBY / FRB);
  if (dt_r == DT_F64)
    k_c27_f64<0, false, double, true><<<g, b64, 0, s>>>(d, wts<double>(A), 0.0, u, b, (double*)r, partials, st);
  else if (dt_r == DT_F32)
    k_c27_f64<0, false, float, true><<<g, b64, 0, s>>>(d, wts<double>(A), 0.0, u, b, (float*)r, partials, st);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_c27_init(const Dims& d, const W27& A, const double* u, const double* b, int dt_r, void* r,
                            double* partials, cudaStream_t s) {
  if (d.g != 1) return cudaErrorInvalidValue;
  const dim3 g = c27_grid(d), b64(CBX, CBY / FRB);
  const int nb = c27_blocks(d);
  if (dt_r == DT_F64)
    k_c27_f64<0, false, double, true, true><<<g, b64, 0, s>>>(d, wts<double>(A), 0.0, u, b, (double*)r, partials, nullptr, nb);
  else if (dt_r == DT_F32)
    k_c27_f64<0, false, float, true, true><<<g, b64, 0, s>>>(d, wts<double>(A), 0.0, u, b, (float*)r, partials, nullptr, nb);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_c27_spai(const Dims& d, const W27& M, double omega, const double* r, double* u,
                            const DevState* st, cudaStream_t s) {
  if (d.g != 1) return cudaErrorInvalidValue;
  k_c27_f64<1, false, double, false><<<c27_grid(d), dim3(CBX, CBY / FRB), 0, s>>>(d, wts<double>(M), omega, r, nullptr,
                                                                                 u, nullptr, st);
  return cudaGetLastError();
}


// ------------------------------------------------------------------ fused FP32 smoothing step
// One SPAI step u' = u - omega M (b - A u) of an inner FP32 level in a single
// pass, out of place (u' goes to another array, so no block reads a value
// that a neighbouring block has already replaced), register-blocked.
//
// A block of GW warps owns a 30 x (GW GR) tile of outputs and a z-chunk;
// warp w owns the strip of GR output rows y0 + GR w .., lane l the column
// x = x0 - 1 + l (lanes 1..30 write; lanes 0 and 31 only supply the
// residual's x-neighbours).  Both stencils are applied through their
// per-plane split (A u)(z) = P(z) + Q(z - 1) + Q(z + 1), P and Q formed from
// the in-plane sums (centre, faces, diagonals) of each plane, so a thread
// carries two numbers per row and plane instead of three sums.  Per plane of
// the z-march each warp
//  - forms P and Q of u(k + 2) on its GR + 2 residual rows from GR + 4 staged
//    u rows, sharing the pair sums u(x-1) + u(x+1) between rows;
//  - forms the residual r(k + 1) = b - (P(k + 1) + (Q(k) + Q(k + 2))) on those
//    rows (zero off the interior);
//  - takes r's x-neighbours by shuffles, forms P and Q of -omega M r(k + 1) on
//    the GR output rows and writes u'(k) = (u(k) + P(k)) + (Q(k - 1) + Q(k + 1)).
// The residual rows next to a strip edge are also formed by the neighbouring
// strip, so warps never exchange residuals.  u (box 40 x (GW GR + 4)) and b
// (box 40 x (GW GR + 2)), both from x = 4 floor((x0 - 2) / 4), arrive by TMA,
// one stage per plane, and plane k stays staged until u'(k) is written (its
// centres); one block barrier per plane returns a stage to the copy engine.
// Traffic is 12 bytes per node instead of 24 for a residual pass followed by a
// SPAI pass; the results equal that route's up to FP32 rounding.
static constexpr int GTX = 30, GBW = 40, GNS = 6;    // output columns, staged row width, stages
// Tile of GW warps x GR output rows per warp: GTY = GW GR rows per block, GRR
// residual rows and GUR u rows per warp, staged boxes of GUH u rows and GBH b rows.
template <int GW, int GR>
struct SmT {
  static constexpr int GTY = GW * GR, GRR = GR + 2, GUR = GR + 4, GUH = GTY + 4, GBH = GTY + 2;
  static constexpr int GUB = GBW * GUH * 4, GBB = GBW * GBH * 4;
  static constexpr int GUBA = (GUB + 127) / 128 * 128, GBBA = (GBB + 127) / 128 * 128;
  static constexpr int GSTAGE = GUBA + GBBA, SMEM = GNS * GSTAGE + GNS * 8;
};

// Per-plane split of a class stencil w on the in-plane sums (C, F, E) of one
// plane: P = w0 C + w1 F + w2 E and Q = w1 C + w2 F + w3 E, so that
// (A u)(z) = P(z) + Q(z - 1) + Q(z + 1).
__device__ __forceinline__ void pq_split(const float (&w)[4], float c, float f, float e, float& P, float& Q) {
  P = fmaf(w[0], c, fmaf(w[1], f, w[2] * e));
  Q = fmaf(w[1], c, fmaf(w[2], f, w[3] * e));
}

// u of one staged plane on the residual rows: P and Q of its in-plane sums
// (the pair sums u(x-1) + u(x+1) shared between rows)
template <int GR>
__device__ __forceinline__ void c27_upq(const float* __restrict__ U, const float (&w)[4], float (&P)[GR + 2],
                                        float (&Q)[GR + 2]) {
  constexpr int GRR = GR + 2, GUR = GR + 4;
  float c[GUR], a[GUR];
#pragma unroll
  for (int s = 0; s < GUR; s++) {
    c[s] = U[s * GBW];
    a[s] = U[s * GBW - 1] + U[s * GBW + 1];
  }
#pragma unroll
  for (int t = 0; t < GRR; t++) pq_split(w, c[t + 1], a[t + 1] + (c[t] + c[t + 2]), a[t] + a[t + 2], P[t], Q[t]);
}

// the residual of one plane on the residual rows: P and Q (of -omega M) of its
// in-plane sums on the output rows, x-neighbours by shuffles
template <int GR>
__device__ __forceinline__ void c27_rpq(const float (&r)[GR + 2], const float (&w)[4], float (&P)[GR], float (&Q)[GR]) {
  constexpr int GRR = GR + 2;
  float ar[GRR];
#pragma unroll
  for (int t = 0; t < GRR; t++) {
    const float l = __shfl_up_sync(0xffffffffu, r[t], 1);
    const float h = __shfl_down_sync(0xffffffffu, r[t], 1);
    ar[t] = l + h;
  }
#pragma unroll
  for (int q = 0; q < GR; q++) pq_split(w, r[q + 1], ar[q + 1] + (r[q] + r[q + 2]), ar[q] + ar[q + 2], P[q], Q[q]);
}

template <int GR>
struct SmoothMarch {
  static constexpr int GRR = GR + 2;
  float up[3][GRR], uq[3][GRR];   // P and Q of u on the residual rows, three planes
  float mp[3][GR], mq[3][GR];     // P and Q of the residual under -omega M on the output rows
};

// RESID: the same march writes the residual r = b - A u of the output rows
// instead (the residual before a restriction), with no M stencil.
template <bool RESID, int GW, int GR>
__global__ void __launch_bounds__(32 * GW, GR <= 4 ? 5 : 3)
    k_c27_smooth(const __grid_constant__ CUtensorMap mU, const __grid_constant__ CUtensorMap mB, Dims d,
                 Wts<float> WA, Wts<float> WM, float om, float* __restrict__ dst, int zc,
                 const DevState* __restrict__ st, int* __restrict__ fault) {
  using T = SmT<GW, GR>;
  constexpr int GTY = T::GTY, GRR = T::GRR, GUB = T::GUB, GBB = T::GBB, GUBA = T::GUBA, GSTAGE = T::GSTAGE;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + GNS * GSTAGE);
  if (st != nullptr && st->done) return;   // uniform
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * GTX + 1, y0b = blockIdx.y * GTY + 1;   // first output node of the tile
  const int xs = ((x0 - 2) >> 2) << 2;                               // box x start, a multiple of 4
  const int k0 = 1 + blockIdx.z * zc, k1 = min(k0 + zc, d.nk() + 1);  // output planes [k0, k1)
  const int zl = k0 - 2, zh = k1 + 1;                                 // staged planes [zl, zh]
  if (tid == 0) {
    for (int q = 0; q < GNS; q++) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int z, int q) {   // thread 0: stage q <- plane z
    if (z > zh) return;
    unsigned char* p = smem + q * GSTAGE;
    unsigned long long* br = &bar[q];
    mbar_expect_tx(br, GUB + GBB);
    tma_load_3d(p, &mU, xs, y0b - 2, z, br);
    tma_load_3d(p + GUBA, &mB, xs, y0b - 1, z, br);
  };
  if (tid == 0)
    for (int q = 0; q < GNS; q++) issue(zl + q, q);
  bool ok = true;
  int wq = 0;
  unsigned wph = 0;
  auto wait_next = [&]() {
    mbar_wait(&bar[wq], wph, ok);
    if (++wq == GNS) { wq = 0; wph ^= 1u; }
  };
  // this lane's residual column and its rows y0w - 1 + t (t = 0 .. GR + 1)
  const int x = x0 - 1 + lane;
  const int y0w = y0b + GR * warp;
  const int col = x - xs;   // box column of x (1 .. 36)
  const bool xin = x >= 1 && x <= d.ni();
  bool rok[GRR];
#pragma unroll
  for (int t = 0; t < GRR; t++) rok[t] = xin && y0w - 1 + t >= 1 && y0w - 1 + t <= d.nj();
  bool oin[GR];
#pragma unroll
  for (int q = 0; q < GR; q++) oin[q] = lane >= 1 && lane <= GTX && x <= d.ni() && y0w + q <= d.nj();
  // stage q's u row y0w - 2 and b row y0w - 1 at column x
  const float* sU = reinterpret_cast<const float*>(smem) + GR * warp * GBW + col;
  const float* sB = reinterpret_cast<const float*>(smem + GUBA) + GR * warp * GBW + col;
  constexpr int SE = GSTAGE / 4;   // stage stride in floats
  float nm[4];   // -omega M
#pragma unroll
  for (int a = 0; a < 4; a++) nm[a] = -om * WM.w[a];
  // residual of plane z on the residual rows: b - (P(z) + (Q(z - 1) + Q(z + 1))), zero off the interior
  auto resid = [&](int z, int q, const float (&Pc)[GRR], const float (&Qm)[GRR], const float (&Qn)[GRR],
                   float (&r)[GRR]) {
    const bool zin = z >= 1 && z <= d.nk();
    const float* B = sB + q * SE;
#pragma unroll
    for (int t = 0; t < GRR; t++) {
      float rv = 0.0f;
      if (zin && rok[t]) rv = B[t * GBW] - (Pc[t] + (Qm[t] + Qn[t]));
      r[t] = rv;
    }
  };
  const long long sy = d.sy(), sz = d.sz();
  float* ob = dst + d.at(min(max(x, 1), d.ni()), min(y0w, d.nj()), k0);   // output row y0w, plane k0
  SmoothMarch<GR> m;
  // prologue: residual planes k0 - 1 and k0 (u planes k0 - 2 .. k0 + 1); u
  // plane z's split sits in slot (z - zl) mod 3, the residual's of plane z in
  // slot (z - k0 + 1) mod 3
  {
    float r[GRR];
    wait_next();
    c27_upq<GR>(sU, WA.w, m.up[0], m.uq[0]);
    wait_next();
    c27_upq<GR>(sU + SE, WA.w, m.up[1], m.uq[1]);
    wait_next();
    c27_upq<GR>(sU + 2 * SE, WA.w, m.up[2], m.uq[2]);
    resid(k0 - 1, 1, m.up[1], m.uq[0], m.uq[2], r);
    c27_rpq<GR>(r, nm, m.mp[0], m.mq[0]);
    wait_next();
    c27_upq<GR>(sU + 3 * SE, WA.w, m.up[0], m.uq[0]);
    resid(k0, 2, m.up[2], m.uq[1], m.uq[0], r);
    if (RESID) {
#pragma unroll
      for (int q = 0; q < GR; q++)
        if (oin[q]) ob[q * sy] = r[q + 1];
    } else {
      c27_rpq<GR>(r, nm, m.mp[1], m.mq[1]);
    }
  }
  __syncthreads();
  if (tid == 0 && ok) {   // planes k0 - 2 and k0 - 1 are no longer read (plane k0 keeps the centres of output k0)
    fence_proxy_async();
    issue(zl + GNS, 0);
    issue(zl + 1 + GNS, 1);
  }
  int s0 = 2, s1 = 3, s2 = 4;   // stages of planes k, k + 1, k + 2 (rotated after every step)
  // output plane k; P = (k - k0) mod 3 fixes the register slots:
  // u splits of planes k, k + 1, k + 2 in slots (P+2)%3, P, (P+1)%3,
  // residual splits of planes k - 1, k, k + 1 in slots P, (P+1)%3, (P+2)%3
  auto step = [&](auto Pc, int k) {
    constexpr int P = decltype(Pc)::value;
    constexpr int UK = (P + 2) % 3, UK1 = P, UK2 = (P + 1) % 3;
    constexpr int RM = P, RC = (P + 1) % 3, RN = (P + 2) % 3;
    wait_next();   // plane k + 2
    c27_upq<GR>(sU + s2 * SE, WA.w, m.up[UK2], m.uq[UK2]);
    float r[GRR];
    resid(k + 1, s1, m.up[UK1], m.uq[UK], m.uq[UK2], r);
    if (RESID) {
      // r of plane k + 1 (plane k0 was written by the prologue)
      ob += sz;
      if (k + 1 < k1)
#pragma unroll
        for (int q = 0; q < GR; q++)
          if (oin[q]) ob[q * sy] = r[q + 1];
    } else {
      c27_rpq<GR>(r, nm, m.mp[RN], m.mq[RN]);
      const float* U = sU + s0 * SE + 2 * GBW;   // u row y0w, plane k
#pragma unroll
      for (int q = 0; q < GR; q++)
        if (oin[q]) ob[q * sy] = (U[q * GBW] + m.mp[RC][q]) + (m.mq[RM][q] + m.mq[RN][q]);
      ob += sz;
    }
    __syncthreads();   // plane k (its u) and plane k + 1 (its b) are no longer read
    if (tid == 0 && ok) {   // after a failed wait no new copy is issued
      fence_proxy_async();
      issue(k + GNS, s0);
    }
    s0 = s1;
    s1 = s2;
    s2 = s2 + 1 == GNS ? 0 : s2 + 1;
  };
  for (int k = k0; k < k1; k += 3) {
    step(std::integral_constant<int, 0>(), k);
    if (k + 1 < k1) step(std::integral_constant<int, 1>(), k + 1);
    if (k + 2 < k1) step(std::integral_constant<int, 2>(), k + 2);
  }
  if (!ok && fault != nullptr) atomicExch(fault, 1);
}

// half_waves: z-chunks enough for about half_waves / 2 waves of blocks
template <bool RESID, int GW, int GR>
static cudaError_t launch_march_t(const Dims& d, const W27& A, const W27& M, double omega, const float* u,
                                  const float* b, float* dst, const DevState* st, int* fault, int half_waves,
                                  cudaStream_t s) {
  using T = SmT<GW, GR>;
  CUtensorMap mu, mb;
  if (!encode_level_map(&mu, DT_F32, u, d, GBW, T::GUH)) return cudaErrorInvalidValue;
  if (!encode_level_map(&mb, DT_F32, b, d, GBW, T::GBH)) return cudaErrorInvalidValue;
  auto kern = k_c27_smooth<RESID, GW, GR>;
  static int blocks_per_sm = 0;
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, 32 * GW, T::SMEM);
    if (e != cudaSuccess) return e;
    blocks_per_sm = std::max(1, blocks_per_sm);
  }
  const int sms = device_sm_count();
  const int gx = (d.ni() + GTX - 1) / GTX, gy = (d.nj() + T::GTY - 1) / T::GTY, nk = d.nk();
  // z-chunks of at least 16 planes (4 extra staged planes each)
  const int want = std::max(1, half_waves * sms * blocks_per_sm / (2 * gx * gy));
  const int zc = std::max(16, (nk + want - 1) / want);
  const dim3 grid(gx, gy, (nk + zc - 1) / zc);
  kern<<<grid, 32 * GW, T::SMEM, s>>>(mu, mb, d, wts<float>(A), wts<float>(M), (float)omega, dst, zc, st, fault);
  return cudaGetLastError();
}

// Tiles: 4 warps x 4 rows (16 rows, 20 warps per SM) below 384 points per side,
// 4 warps x 8 rows (32 rows, residual rows recomputed 1.25 times instead of
// 1.5, 12 warps per SM) above; the same values bit for bit (measured: 255^3
// 0.059 against 0.067 ms, 511^3 0.368 against 0.348 ms per smoothing step).
template <bool RESID>
static cudaError_t launch_march(const Dims& d, const W27& A, const W27& M, double omega, const float* u,
                                const float* b, float* dst, const DevState* st, int* fault, cudaStream_t s) {
  if (d.g != 1 || u == dst) return cudaErrorInvalidValue;
  // measured at 255^3 and 511^3: 8 output rows per warp from 200 points per
  // side (65 thread instructions per node against 90 with 4 rows), with one
  // wave of z-chunks below 384 points and up to 2.5 from 384 (511^3: 3 chunks
  // of 171 planes, 864 blocks; one chunk leaves SMs idle)
  if (d.ni() >= 384 && d.nj() >= 384) return launch_march_t<RESID, 4, 8>(d, A, M, omega, u, b, dst, st, fault, 5, s);
  if (d.ni() >= 200 && d.nj() >= 200) return launch_march_t<RESID, 4, 8>(d, A, M, omega, u, b, dst, st, fault, 2, s);
  return launch_march_t<RESID, 4, 4>(d, A, M, omega, u, b, dst, st, fault, 2, s);
}

cudaError_t launch_c27_smooth(const Dims& d, const W27& A, const W27& M, double omega, const float* u,
                              const float* b, float* dst, const DevState* st, int* fault, cudaStream_t s) {
  return launch_march<false>(d, A, M, omega, u, b, dst, st, fault, s);
}

cudaError_t launch_c27_resid_f32(const Dims& d, const W27& A, const float* u, const float* b, float* r,
                                 const DevState* st, int* fault, cudaStream_t s) {
  return launch_march<true>(d, A, A, 0.0, u, b, r, st, fault, s);
}

// ------------------------------------------------------------------ right-hand side
// f value of node (i, j, k) of the dense layout du, one extrapolated layer on
// every side (cubic along the axis that leaves the array)
__device__ __forceinline__ double f_ext(const Dims& du, const double* __restrict__ rho, int i, int j, int k) {
  const int ni = du.nx, nj = du.ny, nk = du.nz;   // node indices 0..n
  auto at = [&](int a, int b, int c) { return rho[du.at(a, b, c)]; };
  if (i < 0) return 4 * at(0, j, k) - 6 * at(1, j, k) + 4 * at(2, j, k) - at(3, j, k);
  if (i > ni) return 4 * at(ni, j, k) - 6 * at(ni - 1, j, k) + 4 * at(ni - 2, j, k) - at(ni - 3, j, k);
  if (j < 0) return 4 * at(i, 0, k) - 6 * at(i, 1, k) + 4 * at(i, 2, k) - at(i, 3, k);
  if (j > nj) return 4 * at(i, nj, k) - 6 * at(i, nj - 1, k) + 4 * at(i, nj - 2, k) - at(i, nj - 3, k);
  if (k < 0) return 4 * at(i, j, 0) - 6 * at(i, j, 1) + 4 * at(i, j, 2) - at(i, j, 3);
  if (k > nk) return 4 * at(i, j, nk) - 6 * at(i, j, nk - 1) + 4 * at(i, j, nk - 2) - at(i, j, nk - 3);
  return at(i, j, k);
}

// R_h of the compact schemes as a z-march over in-plane sums (the 27-point
// classes of R_h are the classes of A's stencil): per node
//   b = W0 C(z) + W1 (F(z) + C(z-1) + C(z+1)) + W2 (E(z) + F(z-1) + F(z+1))
//     + W3 (sum of the six +-2 offsets)
// with the source scale folded into the weights on the host (no division on
// the device).  As in k_c27_f64 a thread owns FRB consecutive rows of one
// column: per plane it loads the (FRB + 2) x 3 neighbourhood and forms the
// pair sums f(x-1) + f(x+1) once per row; the +-2 offsets in y come from those
// rows where they lie inside them, in z from the centres of planes k - 2 and
// k + 2 kept or prefetched in registers, and past the node array from the
// cubic extrapolation (f_ext).
template <int ORDER>
__global__ void __launch_bounds__(CBX*(CBY / FRB))
    k_c27_rhs(Dims d, Dims du, const double* __restrict__ rho, Wts<double> W, double* __restrict__ b) {
  const int i = blockIdx.x * CBX + threadIdx.x + 1;
  const int j0 = blockIdx.y * CBY + threadIdx.y * FRB + 1;   // rows j0 .. j0 + FRB - 1
  const int k0 = blockIdx.z * CZC + 1, k1 = min(k0 + CZC, d.nk() + 1);
  if (i > d.ni() || j0 > d.nj()) return;
  const long long sy = du.sy(), sz = du.sz();
  if (ORDER == 2) {
    for (int k = k0; k < k1; k++)
#pragma unroll
      for (int q = 0; q < FRB; q++)
        if (j0 + q <= d.nj()) b[d.at(i, j0 + q, k)] = W.w[0] * rho[du.at(i, j0 + q, k)];
    return;
  }
  const int ny = du.ny, nz = du.nz;   // last node index along y and z
  // rows j0 - 1 + s of the node array, clamped to it: a clamped row only
  // feeds rows that are not written
  long long roff[FRB + 2];
#pragma unroll
  for (int s = 0; s < FRB + 2; s++) roff[s] = (long long)min(j0 - 1 + s, ny) * sy + i;
  auto load = [&](int k, double (&v)[FRB + 2][3]) {
    const double* p = rho + (long long)k * sz;
#pragma unroll
    for (int s = 0; s < FRB + 2; s++) {
      v[s][0] = p[roff[s] - 1];
      v[s][1] = p[roff[s]];
      v[s][2] = p[roff[s] + 1];
    }
  };
  auto sums = [&](const double (&v)[FRB + 2][3], double (&C)[FRB], double (&F)[FRB], double (&E)[FRB]) {
    double a[FRB + 2];
#pragma unroll
    for (int s = 0; s < FRB + 2; s++) a[s] = v[s][0] + v[s][2];
#pragma unroll
    for (int q = 0; q < FRB; q++) {
      C[q] = v[q + 1][1];
      F[q] = a[q + 1] + (v[q][1] + v[q + 2][1]);
      E[q] = a[q] + a[q + 2];
    }
  };
  const bool side_x = i == 1 || i == d.ni();   // x offsets +-2 leave the array
  double v[FRB + 2][3], vn[FRB + 2][3];
  double Cm[FRB], Fm[FRB], Cc[FRB], Fc[FRB], Ec[FRB], cm2[FRB];
  {
    double Em[FRB];
    load(k0 - 1, v);
    sums(v, Cm, Fm, Em);
  }
  load(k0, v);
  sums(v, Cc, Fc, Ec);
  double Sc[FRB + 2];   // centres of the loaded rows of plane k (for the y offsets +-2)
#pragma unroll
  for (int s = 0; s < FRB + 2; s++) Sc[s] = v[s][1];
  if (ORDER == 6)
#pragma unroll
    for (int q = 0; q < FRB; q++) cm2[q] = f_ext(du, rho, i, min(j0 + q, d.nj()), k0 - 2);   // centres of plane k0 - 2
  load(k0 + 1, v);
  for (int k = k0; k < k1; k++) {
    if (k + 2 <= nz) load(k + 2, vn);   // issued before the arithmetic of plane k
    double Cn[FRB], Fn[FRB], En[FRB];
    sums(v, Cn, Fn, En);
    const double* p = rho + (long long)k * sz;
#pragma unroll
    for (int q = 0; q < FRB; q++) {
      // rows past nj are not written; their offsets use row nj so that f_ext
      // only ever extrapolates along one axis
      const int j = min(j0 + q, d.nj());
      const double fa = Fc[q] + (Cm[q] + Cn[q]);
      double val;
      if (ORDER == 4) {
        val = fma(W.w[0], Cc[q], W.w[1] * fa);
      } else {
        const double ed = Ec[q] + (Fm[q] + Fn[q]);
        double xs;
        if (side_x) xs = f_ext(du, rho, i - 2, j, k) + f_ext(du, rho, i + 2, j, k);
        else xs = p[roff[q + 1] - 2] + p[roff[q + 1] + 2];
        // y - 2 is loaded row q - 1 for q >= 1, y + 2 loaded row q + 3 for q + 3 <= FRB + 1
        double ym2, yp2;
        if (q >= 1) ym2 = Sc[q - 1];
        else ym2 = j - 2 >= 0 ? p[(long long)(j - 2) * sy + i] : f_ext(du, rho, i, j - 2, k);
        if (j + 2 > ny) yp2 = f_ext(du, rho, i, j + 2, k);
        else if (q + 3 <= FRB + 1) yp2 = Sc[q + 3];
        else yp2 = p[(long long)(j + 2) * sy + i];
        const double ys = ym2 + yp2;
        const double cp2 = k + 2 <= nz ? vn[q + 1][1] : f_ext(du, rho, i, j, k + 2);
        const double ax = (xs + ys) + (cm2[q] + cp2);
        val = fma(W.w[0], Cc[q], fma(W.w[1], fa, fma(W.w[2], ed, W.w[3] * ax)));
        cm2[q] = Cm[q];
      }
      if (j0 + q <= d.nj()) b[d.at(i, j, k)] = val;
      Cm[q] = Cc[q];
      Fm[q] = Fc[q];
      Cc[q] = Cn[q];
      Fc[q] = Fn[q];
      Ec[q] = En[q];
    }
#pragma unroll
    for (int s = 0; s < FRB + 2; s++) {
      Sc[s] = v[s][1];
#pragma unroll
      for (int c = 0; c < 3; c++) v[s][c] = vn[s][c];
    }
  }
}

cudaError_t launch_c27_rhs(const Dims& d, const Dims& du, int order, const double* rho, double fscale,
                           double* b, cudaStream_t s) {
  if (d.g != 1 || du.g != 1) return cudaErrorInvalidValue;
  if (order == 6 && (d.nx < 4 || d.ny < 4 || d.nz < 4)) return cudaErrorInvalidValue;
  const dim3 g = c27_grid(d), blk(CBX, CBY / FRB);
  // R_h weights per class (centre, faces, edges, +-2 offsets) times the source scale
  if (order == 2) {
    k_c27_rhs<2><<<g, blk, 0, s>>>(d, du, rho, Wts<double>{{fscale, 0.0, 0.0, 0.0}}, b);
  } else if (order == 4) {
    k_c27_rhs<4><<<g, blk, 0, s>>>(d, du, rho, Wts<double>{{fscale * 0.5, fscale / 12.0, 0.0, 0.0}}, b);
  } else {
    k_c27_rhs<6><<<g, blk, 0, s>>>(
        d, du, rho, Wts<double>{{fscale * (67.0 / 120.0), fscale / 18.0, fscale / 90.0, -fscale / 240.0}}, b);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ coarsest level
// CG on -A u = -b from u = 0 (A negative definite), one CTA: x, r, q over the
// unknowns and p over all nodes (zero boundary) in shared memory.
static constexpr int CCG_THREADS = 1024;

__device__ double ccg_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[32] = t;
  __syncthreads();
  return red[32];
}

template <typename T>
__global__ void __launch_bounds__(CCG_THREADS)
    k_c27_coarse_cg(Dims d, W27 A, const T* __restrict__ b, T* __restrict__ u, double tol,
                    const DevState* __restrict__ st) {
  if (st != nullptr && st->done) return;
  extern __shared__ double sm[];
  const int nx = d.nx + 1, ny = d.ny + 1, nz = d.nz + 1;   // nodes per axis
  const int nn = nx * ny * nz;
  const int ni = d.ni(), nj = d.nj(), nk = d.nk(), nu = ni * nj * nk;
  double* p = sm;              // [nn] all nodes, boundary zero
  double* x = p + nn;          // [nu]
  double* r = x + nu;
  double* q = r + nu;
  double* red = q + nu;        // [33]
  auto node = [&](int t) {     // unknown t -> node index in p
    const int i = t % ni + 1, j = (t / ni) % nj + 1, k = t / (ni * nj) + 1;
    return (k * ny + j) * nx + i;
  };
  auto gidx = [&](int t) {
    const int i = t % ni + 1, j = (t / ni) % nj + 1, k = t / (ni * nj) + 1;
    return d.at(i, j, k);
  };
  for (int t = threadIdx.x; t < nn; t += blockDim.x) p[t] = 0.0;
  __syncthreads();
  double loc = 0.0;
  for (int t = threadIdx.x; t < nu; t += blockDim.x) {
    const double v = -(double)b[gidx(t)];
    x[t] = 0.0;
    r[t] = v;
    p[node(t)] = v;
    loc = fma(v, v, loc);
  }
  double rr = ccg_sum(loc, red);
  const double ref = sqrt(rr) > 0.0 ? sqrt(rr) : 1.0;
  const int sy = nx, sz = nx * ny;
  for (int it = 0; it < nu && sqrt(rr) / ref > tol; it++) {
    loc = 0.0;
    for (int t = threadIdx.x; t < nu; t += blockDim.x) {
      const int c = node(t);
      const double f = (p[c - 1] + p[c + 1]) + (p[c - sy] + p[c + sy]) + (p[c - sz] + p[c + sz]);
      const double e = ((p[c - sy - 1] + p[c - sy + 1]) + (p[c + sy - 1] + p[c + sy + 1])) +
                       ((p[c - sz - 1] + p[c - sz + 1]) + (p[c + sz - 1] + p[c + sz + 1])) +
                       ((p[c - sz - sy] + p[c - sz + sy]) + (p[c + sz - sy] + p[c + sz + sy]));
      const double k8 = ((p[c - sz - sy - 1] + p[c - sz - sy + 1]) + (p[c - sz + sy - 1] + p[c - sz + sy + 1])) +
                        ((p[c + sz - sy - 1] + p[c + sz - sy + 1]) + (p[c + sz + sy - 1] + p[c + sz + sy + 1]));
      const double v = -(A.w[0] * p[c] + A.w[1] * f + A.w[2] * e + A.w[3] * k8);
      q[t] = v;
      loc = fma(p[c], v, loc);
    }
    const double pq = ccg_sum(loc, red);
    const double alpha = rr / pq;
    loc = 0.0;
    for (int t = threadIdx.x; t < nu; t += blockDim.x) {
      x[t] = fma(alpha, p[node(t)], x[t]);
      const double v = fma(-alpha, q[t], r[t]);
      r[t] = v;
      loc = fma(v, v, loc);
    }
    const double rn = ccg_sum(loc, red);
    const double beta = rn / rr;
    rr = rn;
    for (int t = threadIdx.x; t < nu; t += blockDim.x) {
      const int c = node(t);
      p[c] = fma(beta, p[c], r[t]);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nu; t += blockDim.x) u[gidx(t)] = (T)x[t];
}

size_t c27_coarse_smem(const Dims& d) {
  const size_t nn = (size_t)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  const size_t nu = (size_t)d.ni() * d.nj() * d.nk();
  return (nn + 3 * nu + 33) * sizeof(double);
}

template <typename T>
static cudaError_t coarse_cg_t(const Dims& d, const W27& A, const T* b, T* u, double tol, const DevState* st,
                               cudaStream_t s) {
  const size_t smem = c27_coarse_smem(d);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  static size_t opted = 0;
  if (smem > 48 * 1024 && smem > opted) {
    cudaError_t e = cudaFuncSetAttribute(k_c27_coarse_cg<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    opted = smem;
  }
  k_c27_coarse_cg<T><<<1, CCG_THREADS, smem, s>>>(d, A, b, u, tol, st);
  return cudaGetLastError();
}

cudaError_t launch_c27_coarse_cg(const Dims& d, const W27& A, const double* b, double* u, double tol,
                                 const DevState* st, cudaStream_t s) {
  return coarse_cg_t<double>(d, A, b, u, tol, st, s);
}

cudaError_t launch_c27_coarse_cg_dt(const Dims& d, const W27& A, int dt, const void* b, void* u, double tol,
                                    const DevState* st, cudaStream_t s) {
  if (dt == DT_F64) return coarse_cg_t<double>(d, A, (const double*)b, (double*)u, tol, st, s);
  if (dt == DT_F32) return coarse_cg_t<float>(d, A, (const float*)b, (float*)u, tol, st, s);
  return cudaErrorInvalidValue;
}

}  // namespace ps
