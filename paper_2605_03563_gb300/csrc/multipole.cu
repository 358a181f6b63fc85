// Multipole open boundary on Cartesian grids (Sec. 2.2).
//
// Moments (Eq. outer_multipole) with the Schmidt-normalised regular solid
// harmonics R_lm = sqrt(4 pi/(2l+1)) r^l Y_lm, which are homogeneous
// polynomials of degree l in (x, y, z).  The GPU therefore reduces the density
// to Cartesian monomial moments M_abc = sum rho dV x^a y^b z^c (a+b+c <= l_max)
// in three separable passes -- x along rows, y within planes, z across planes --
// and maps them to q_lm with a fixed sparse table built on the host.  The
// per-node cost is l_max+1 FP64 multiply-adds and one read of rho.
//
// Boundary values (Eq. outer_expansion): Phi = -G sum_lm q_lm R_lm(x) / r^(2l+1),
// with R_lm evaluated per node from the recurrences
//   (x + i y)^m = C_m + i S_m,
//   T_mm = (2m-1)!!,  T_{m+1,m} = (2m+1) z T_mm,
//   (l-m) T_lm = (2l-1) z T_{l-1,m} - (l+m-1) r^2 T_{l-2,m},
//   R_l0 = T_l0,  R_l(+-m) = sqrt(2 (l-m)!/(l+m)!) T_lm {C_m, S_m}
// (T_lm = r^l P_l^m(cos t) / (r sin t)^m, P without the Condon-Shortley phase).
#include <cmath>
#include <map>

#include "multipole.cuh"

namespace ps {

static constexpr int MAXL = 16;

// ------------------------------------------------------------------ host tables
namespace {
using Poly = std::map<int, double>;  // key = (a*(L+1)+b)*(L+1)+c

struct PolyAlg {
  int L;
  int key(int a, int b, int c) const { return (a * (L + 1) + b) * (L + 1) + c; }
  void split(int k, int& a, int& b, int& c) const {
    c = k % (L + 1);
    b = (k / (L + 1)) % (L + 1);
    a = k / ((L + 1) * (L + 1));
  }
  Poly mul_var(const Poly& p, int var) const {
    Poly out;
    for (auto& kv : p) {
      int a, b, c;
      split(kv.first, a, b, c);
      if (var == 0) a++;
      else if (var == 1) b++;
      else c++;
      out[key(a, b, c)] += kv.second;
    }
    return out;
  }
  Poly mul(const Poly& p, const Poly& q) const {
    Poly out;
    for (auto& u : p)
      for (auto& v : q) {
        int a1, b1, c1, a2, b2, c2;
        split(u.first, a1, b1, c1);
        split(v.first, a2, b2, c2);
        out[key(a1 + a2, b1 + b2, c1 + c2)] += u.second * v.second;
      }
    return out;
  }
  static Poly axpy(double a, const Poly& x, double b, const Poly& y) {
    Poly out;
    for (auto& kv : x) out[kv.first] += a * kv.second;
    for (auto& kv : y) out[kv.first] += b * kv.second;
    return out;
  }
};

double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; i++) f *= i;
  return f;
}
}  // namespace

void build_multipole_tables(int L, MultipoleTables* t) {
  t->lmax = L;
  const int W = L + 1;
  t->rec_a.assign(W * W, 0.0);
  t->rec_b.assign(W * W, 0.0);
  t->nrm.assign(W * W, 0.0);
  t->dfac.assign(W, 1.0);
  for (int m = 1; m <= L; m++) t->dfac[m] = t->dfac[m - 1] * (2 * m - 1);
  for (int l = 0; l <= L; l++)
    for (int m = 0; m <= l; m++) {
      if (l >= m + 2) {
        t->rec_a[l * W + m] = (double)(2 * l - 1) / (double)(l - m);
        t->rec_b[l * W + m] = (double)(l + m - 1) / (double)(l - m);
      }
      t->nrm[l * W + m] = m == 0 ? 1.0 : std::sqrt(2.0 * factorial(l - m) / factorial(l + m));
    }
  // polynomials
  PolyAlg A{L};
  std::vector<Poly> Cm(W), Sm(W);
  Cm[0][A.key(0, 0, 0)] = 1.0;
  for (int m = 0; m < L; m++) {
    Cm[m + 1] = PolyAlg::axpy(1.0, A.mul_var(Cm[m], 0), -1.0, A.mul_var(Sm[m], 1));
    Sm[m + 1] = PolyAlg::axpy(1.0, A.mul_var(Sm[m], 0), 1.0, A.mul_var(Cm[m], 1));
  }
  Poly r2;
  r2[A.key(2, 0, 0)] = 1.0;
  r2[A.key(0, 2, 0)] = 1.0;
  r2[A.key(0, 0, 2)] = 1.0;
  std::vector<Poly> R(W * W);
  for (int m = 0; m <= L; m++) {
    std::vector<Poly> T(W);
    T[m][A.key(0, 0, 0)] = t->dfac[m];
    if (m + 1 <= L) {
      Poly z1 = A.mul_var(T[m], 2);
      T[m + 1] = PolyAlg::axpy(2.0 * m + 1.0, z1, 0.0, Poly());
    }
    for (int l = m + 2; l <= L; l++)
      T[l] = PolyAlg::axpy(t->rec_a[l * W + m], A.mul_var(T[l - 1], 2), -t->rec_b[l * W + m],
                           A.mul(r2, T[l - 2]));
    for (int l = m; l <= L; l++) {
      double n = t->nrm[l * W + m];
      if (m == 0) {
        R[l * l + l] = T[l];
      } else {
        R[l * l + l + m] = PolyAlg::axpy(n, A.mul(T[l], Cm[m]), 0.0, Poly());
        R[l * l + l - m] = PolyAlg::axpy(n, A.mul(T[l], Sm[m]), 0.0, Poly());
      }
    }
  }
  t->off.assign(W * W + 1, 0);
  t->mono.clear();
  t->val.clear();
  for (int lm = 0; lm < W * W; lm++) {
    t->off[lm] = (int)t->mono.size();
    for (auto& kv : R[lm]) {
      if (kv.second == 0.0) continue;
      t->mono.push_back(kv.first);
      t->val.push_back(kv.second);
    }
  }
  t->off[W * W] = (int)t->mono.size();
}

// ------------------------------------------------------------------ moment kernels
// Pass 1: x-row moments.  One warp per row (4 rows per warp, 8 warps per block);
// the powers x_i^a (a <= L) of the block's rows come from a shared table when
// it fits (one FP64 FMA per node and power), else from a running product.
constexpr int ROWS_PER_BLOCK = 32;

template <int L, bool TABLE>
__global__ void __launch_bounds__(256)
    k_mp_rows(Dims d, double x0, double hx, double dV, const double* __restrict__ rho,
              double* __restrict__ rowmom) {
  extern __shared__ double X[];   // [(L+1) * ni] when TABLE
  const int ni = d.ni();
  if (TABLE) {
    for (int t = threadIdx.x; t < ni; t += blockDim.x) {
      const double x = fma((double)(t + 1), hx, x0);
      double p = 1.0;
#pragma unroll
      for (int a = 0; a <= L; a++) {
        X[a * ni + t] = p;
        p *= x;
      }
    }
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrows = d.nj() * d.nk();
  const int g = d.g;
  for (int q = 0; q < ROWS_PER_BLOCK / 8; q++) {
    const int u = blockIdx.x * ROWS_PER_BLOCK + q * 8 + warp;   // row id = k * nj + j
    if (u >= nrows) break;
    const int j = u % d.nj(), k = u / d.nj();
    const long long row = d.at(g, j + g, k + g);
    double s[L + 1];
#pragma unroll
    for (int a = 0; a <= L; a++) s[a] = 0.0;
    for (int i = lane; i < ni; i += 32) {
      const double w = rho[row + i] * dV;
      if (TABLE) {
#pragma unroll
        for (int a = 0; a <= L; a++) s[a] = fma(w, X[a * ni + i], s[a]);
      } else {
        const double x = fma((double)(i + 1), hx, x0);
        double p = w;
#pragma unroll
        for (int a = 0; a <= L; a++) {
          s[a] += p;
          p *= x;
        }
      }
    }
#pragma unroll
    for (int a = 0; a <= L; a++) {
      const double v = warp_sum(s[a]);
      if (lane == 0) rowmom[(long long)u * (L + 1) + a] = v;
    }
  }
}

__device__ __forceinline__ int pair_index(int a, int b, int L) {
  // pairs (a, b) with a + b <= L ordered by a, then b
  return a * (L + 1) - a * (a - 1) / 2 + b;
}

// Pass 2: y-moments within each plane.  One block per plane; warp w handles
// pairs w, w+8, ...; lanes stride over the rows; y^b from a shared table.
__global__ void __launch_bounds__(256)
    k_mp_planes(Dims d, double y0, double hy, int L, const double* __restrict__ rowmom,
                double* __restrict__ planemom) {
  extern __shared__ double Y[];   // [(L+1) * nj]
  const int nj = d.nj(), k = blockIdx.x;
  for (int t = threadIdx.x; t < nj; t += blockDim.x) {
    const double y = fma((double)(t + 1), hy, y0);
    double p = 1.0;
    for (int b = 0; b <= L; b++) {
      Y[b * nj + t] = p;
      p *= y;
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P2 = (L + 1) * (L + 2) / 2;
  for (int t = warp; t < P2; t += 8) {
    int a = 0, rem = t;
    while (rem > L - a) { rem -= L - a + 1; a++; }
    const int b = rem;
    double acc = 0.0;
    for (int j = lane; j < nj; j += 32)
      acc = fma(rowmom[((long long)k * nj + j) * (L + 1) + a], Y[b * nj + j], acc);
    acc = warp_sum(acc);
    if (lane == 0) planemom[(long long)k * P2 + pair_index(a, b, L)] = acc;
  }
}

// Pass 3: z-moments across planes (warp per monomial, lanes over planes),
// then the sparse map from monomials to q_lm.
__global__ void __launch_bounds__(1024)
    k_mp_final(Dims d, double z0, double hz, int L, const double* __restrict__ planemom,
               const int* __restrict__ off, const int* __restrict__ mono,
               const double* __restrict__ val, double* __restrict__ q) {
  extern __shared__ double M[];   // (L+1)^3
  const int W = L + 1;
  const int P2 = W * (W + 1) / 2;
  const int nk = d.nk();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = threadIdx.x; t < W * W * W; t += blockDim.x) M[t] = 0.0;
  __syncthreads();
  for (int t = warp; t < W * W * W; t += nw) {
    const int c = t % W, b = (t / W) % W, a = t / (W * W);
    if (a + b + c > L) continue;
    const int pi = pair_index(a, b, L);
    double acc = 0.0;
    for (int k = lane; k < nk; k += 32) {
      const double z = fma((double)(k + 1), hz, z0);
      double zc = 1.0;
      for (int e = 0; e < c; e++) zc *= z;
      acc = fma(planemom[(long long)k * P2 + pi], zc, acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) M[t] = acc;
  }
  __syncthreads();
  for (int lm = threadIdx.x; lm < W * W; lm += blockDim.x) {
    double acc = 0.0;
    for (int t = off[lm]; t < off[lm + 1]; t++) acc = fma(val[t], M[mono[t]], acc);
    q[lm] = acc;
  }
}

// ------------------------------------------------------------------ boundary values
__device__ double eval_expansion(double x, double y, double z, int L, const double* __restrict__ q,
                                 const double* __restrict__ consts, double G) {
  const int W = L + 1;
  const double* rec_a = consts;
  const double* rec_b = consts + W * W;
  const double* nrm = consts + 2 * W * W;
  const double* dfac = consts + 3 * W * W;
  const double r2 = x * x + y * y + z * z;
  double acc[MAXL + 1];
  for (int l = 0; l <= L; l++) acc[l] = 0.0;
  double Cm = 1.0, Sm = 0.0;
  for (int m = 0; m <= L; m++) {
    if (m > 0) {
      const double c = x * Cm - y * Sm;
      Sm = x * Sm + y * Cm;
      Cm = c;
    }
    double t2 = 0.0, t1 = dfac[m];   // T_{l-2,m}, T_{l-1,m}
    for (int l = m; l <= L; l++) {
      double T;
      if (l == m) T = dfac[m];
      else if (l == m + 1) T = (2.0 * m + 1.0) * z * t1;
      else T = rec_a[l * W + m] * z * t1 - rec_b[l * W + m] * r2 * t2;
      if (l > m) { t2 = t1; t1 = T; }
      const double ang = m == 0 ? q[l * l + l] : fma(q[l * l + l + m], Cm, q[l * l + l - m] * Sm);
      acc[l] = fma(nrm[l * W + m] * T, ang, acc[l]);
    }
  }
  const double ir = 1.0 / sqrt(r2);
  const double ir2 = ir * ir;
  double f = ir, phi = 0.0;
  for (int l = 0; l <= L; l++) {
    phi = fma(acc[l], f, phi);
    f *= ir2;
  }
  return -G * phi;
}

__global__ void __launch_bounds__(256)
    k_mp_faces(Dims d, double x0, double y0, double z0, double hx, double hy, double hz, int L,
               double G, const double* __restrict__ q, const double* __restrict__ consts,
               double* __restrict__ phi) {
  const long long id0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int g = d.g, ni = d.ni(), nj = d.nj(), nk = d.nk();
  const long long nzs = (long long)g * d.ex * d.ey;     // one z slab
  const long long nys = (long long)g * d.ex * nk;       // one y slab
  const long long nxs = (long long)g * nj * nk;         // one x slab
  const long long total = 2 * (nzs + nys + nxs);
  if (id0 >= total) return;
  long long id = id0;
  int i, j, k;
  if (id < 2 * nzs) {
    const int s = (int)(id / nzs);
    const long long rem = id % nzs;
    i = (int)(rem % d.ex);
    j = (int)((rem / d.ex) % d.ey);
    const int kk = (int)(rem / ((long long)d.ex * d.ey));
    k = s == 0 ? kk : g + nk + kk;
  } else if ((id -= 2 * nzs) < 2 * nys) {
    const int s = (int)(id / nys);
    const long long rem = id % nys;
    i = (int)(rem % d.ex);
    const long long t = rem / d.ex;
    const int jj = (int)(t % g);
    k = g + (int)(t / g);
    j = s == 0 ? jj : g + nj + jj;
  } else {
    id -= 2 * nys;
    const int s = (int)(id / nxs);
    const long long rem = id % nxs;
    const int ii = (int)(rem % g);
    const long long t = rem / g;
    j = g + (int)(t % nj);
    k = g + (int)(t / nj);
    i = s == 0 ? ii : g + ni + ii;
  }
  const double x = fma((double)(i - g + 1), hx, x0);
  const double y = fma((double)(j - g + 1), hy, y0);
  const double z = fma((double)(k - g + 1), hz, z0);
  phi[d.at(i, j, k)] = eval_expansion(x, y, z, L, q, consts, G);
}

// ------------------------------------------------------------------ host launchers
cudaError_t cart_multipole_alloc(const Dims& d, int lmax, const MultipoleTables& t,
                                 CartMultipoleDev* m) {
  const int W = lmax + 1;
  m->lmax = lmax;
  size_t nrow = (size_t)d.nj() * d.nk() * W;
  size_t nplane = (size_t)d.nk() * W * (W + 1) / 2;
  size_t ncons = 3 * (size_t)W * W + W;
  cudaError_t e;
  if ((e = cudaMalloc(&m->rowmom, nrow * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->planemom, nplane * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->q, (size_t)W * W * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->off, t.off.size() * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->mono, std::max<size_t>(1, t.mono.size()) * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->val, std::max<size_t>(1, t.val.size()) * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->consts, ncons * sizeof(double))) != cudaSuccess) return e;
  m->bytes = (nrow + nplane + W * W + ncons + t.val.size()) * sizeof(double) +
             (t.off.size() + t.mono.size()) * sizeof(int);
  std::vector<double> cons;
  cons.insert(cons.end(), t.rec_a.begin(), t.rec_a.end());
  cons.insert(cons.end(), t.rec_b.begin(), t.rec_b.end());
  cons.insert(cons.end(), t.nrm.begin(), t.nrm.end());
  cons.insert(cons.end(), t.dfac.begin(), t.dfac.end());
  if ((e = cudaMemcpy(m->off, t.off.data(), t.off.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if (!t.mono.empty()) {
    if ((e = cudaMemcpy(m->mono, t.mono.data(), t.mono.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(m->val, t.val.data(), t.val.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  }
  return cudaMemcpy(m->consts, cons.data(), cons.size() * sizeof(double), cudaMemcpyHostToDevice);
}

void cart_multipole_free(CartMultipoleDev* m) {
  cudaFree(m->rowmom);
  cudaFree(m->planemom);
  cudaFree(m->q);
  cudaFree(m->off);
  cudaFree(m->mono);
  cudaFree(m->val);
  cudaFree(m->consts);
  *m = CartMultipoleDev();
}

template <int L>
static void rows_launch(const Dims& d, double x0, double hx, double dV, const double* rho,
                        double* rowmom, cudaStream_t s) {
  const int nrows = d.nj() * d.nk();
  const unsigned blocks = (nrows + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
  const size_t table = (size_t)(L + 1) * d.ni() * sizeof(double);
  if (table <= 48 * 1024)
    k_mp_rows<L, true><<<blocks, 256, table, s>>>(d, x0, hx, dV, rho, rowmom);
  else
    k_mp_rows<L, false><<<blocks, 256, 0, s>>>(d, x0, hx, dV, rho, rowmom);
}

cudaError_t launch_cart_moments(const Dims& d, const double lo[3], const double h[3],
                                const double origin[3], const double* rho, CartMultipoleDev* m,
                                cudaStream_t s) {
  const int L = m->lmax;
  if (L < 0 || L > MAXL) return cudaErrorInvalidValue;
  if ((size_t)(L + 1) * d.nj() * sizeof(double) > 48 * 1024) return cudaErrorInvalidValue;
  const double dV = h[0] * h[1] * h[2];
  const double x0 = lo[0] - origin[0];
  switch (L) {
    case 0: rows_launch<0>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 1: rows_launch<1>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 2: rows_launch<2>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 3: rows_launch<3>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 4: rows_launch<4>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 5: rows_launch<5>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 6: rows_launch<6>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 7: rows_launch<7>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 8: rows_launch<8>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 9: rows_launch<9>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 10: rows_launch<10>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 11: rows_launch<11>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 12: rows_launch<12>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 13: rows_launch<13>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 14: rows_launch<14>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    case 15: rows_launch<15>(d, x0, h[0], dV, rho, m->rowmom, s); break;
    default: rows_launch<16>(d, x0, h[0], dV, rho, m->rowmom, s); break;
  }
  const size_t ytab = (size_t)(L + 1) * d.nj() * sizeof(double);
  k_mp_planes<<<d.nk(), 256, ytab, s>>>(d, lo[1] - origin[1], h[1], L, m->rowmom, m->planemom);
  const int W = L + 1;
  size_t smem = (size_t)W * W * W * sizeof(double);
  k_mp_final<<<1, 1024, smem, s>>>(d, lo[2] - origin[2], h[2], L, m->planemom, m->off, m->mono,
                                   m->val, m->q);
  return cudaGetLastError();
}

cudaError_t launch_cart_faces(const Dims& d, const double lo[3], const double h[3],
                              const double origin[3], double G, const double* q,
                              const CartMultipoleDev* m, double* phi, cudaStream_t s) {
  const long long total = 2LL * d.g * ((long long)d.ex * d.ey + (long long)d.ex * d.nk() +
                                       (long long)d.nj() * d.nk());
  const int thr = 256;
  const long long blocks = (total + thr - 1) / thr;
  k_mp_faces<<<(unsigned)blocks, thr, 0, s>>>(d, lo[0] - origin[0], lo[1] - origin[1],
                                              lo[2] - origin[2], h[0], h[1], h[2], m->lmax, G, q,
                                              m->consts, phi);
  return cudaGetLastError();
}

}  // namespace ps
