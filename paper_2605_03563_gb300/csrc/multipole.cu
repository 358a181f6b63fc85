// Multipole open boundary on Cartesian grids (Sec. 2.2).
//
// Moments (Eq. outer_multipole) with the Schmidt-normalised regular solid
// harmonics R_lm = sqrt(4 pi/(2l+1)) r^l Y_lm, which are homogeneous
// polynomials of degree l in (x, y, z).  The GPU therefore reduces the density
// to Cartesian monomial moments M_abc = sum rho dV x^a y^b z^c (a+b+c <= l_max)
// in three separable passes -- z along columns, then y, then x -- and maps them
// to q_lm with a fixed sparse table built on the host.  The per-node cost is
// l_max+1 FP64 multiply-adds and one coalesced read of rho.
//
// Boundary values (Eq. outer_expansion): Phi = -G sum_lm q_lm R_lm(x) / r^(2l+1).
// P_l = sum_m q_lm R_lm is a homogeneous polynomial of degree l with
// coefficients C_abc (a+b+c = l), formed once per solve from q and the table.
// Since r^-(2l+1) x^a y^b z^c = (1/r) (x/r^2)^a (y/r^2)^b (z/r^2)^c, the sum
// over l is one polynomial of total degree <= l_max in (x, y, z)/r^2:
//   Phi = -G (1/r) F(x/r^2, y/r^2, z/r^2),  F(u, v, w) = sum C_abc u^a v^b w^c,
// evaluated per node by nested Horner, one FMA per coefficient.  The table
// of R_lm's monomials is built on the host from the recurrences
//   (x + i y)^m = C_m + i S_m,
//   T_mm = (2m-1)!!,  T_{m+1,m} = (2m+1) z T_mm,
//   (l-m) T_lm = (2l-1) z T_{l-1,m} - (l+m-1) r^2 T_{l-2,m},
//   R_l0 = T_l0,  R_l(+-m) = sqrt(2 (l-m)!/(l+m)!) T_lm {C_m, S_m}
// (T_lm = r^l P_l^m(cos t) / (r sin t)^m, P without the Condon-Shortley phase).
#include <algorithm>
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
  // transpose: for every monomial slot, its (lm, val) pairs in increasing lm
  const int NS = W * W * W;
  t->toff.assign(NS + 1, 0);
  for (int e = 0; e < (int)t->mono.size(); e++) t->toff[t->mono[e] + 1]++;
  for (int q = 0; q < NS; q++) t->toff[q + 1] += t->toff[q];
  t->tlm.assign(t->mono.size(), 0);
  t->tval.assign(t->mono.size(), 0.0);
  std::vector<int> fill(t->toff.begin(), t->toff.end() - 1);
  for (int lm = 0; lm < W * W; lm++)
    for (int e = t->off[lm]; e < t->off[lm + 1]; e++) {
      const int slot = fill[t->mono[e]]++;
      t->tlm[slot] = lm;
      t->tval[slot] = t->val[e];
    }
}

// ------------------------------------------------------------------ moment kernels
// Pass 1: z-moments of every (i, j) column, S_c(i, j) = sum_k rho(i, j, k) z_k^c,
// c <= L.  One thread per column and z-chunk: a warp reads 32 consecutive x
// nodes of a plane (coalesced).  The chunk's planes are taken in pairs
// symmetric about its centre z_m, z = z_m +- u: the pair adds
// (rho_hi + rho_lo) u^c to the moment about z_m for even c and
// (rho_hi - rho_lo) u^c for odd c, (L+3)/2 FP64 instructions per node instead
// of L+1 (the middle plane of an odd chunk adds to c = 0 only); the moments
// about z_m move to the origin once per column by the binomial expansion
// sum_e C(c, e) z_m^(c-e) mu_e.  No reduction is needed inside the pass;
// z-chunks (for parallelism on small grids) leave separate partial sums that
// pass 2 adds up.
constexpr int MP_KC_MAX = 256;   // planes per z-chunk

template <int L>
__global__ void __launch_bounds__(256)
    k_mp_cols(Dims d, double z0, double hz, int kc, const double* __restrict__ rho,
              double* __restrict__ colmom) {
  __shared__ double U[MP_KC_MAX / 2 * (L + 1)];   // u_t^c of the chunk's plane pairs
  __shared__ double Wsh[(L + 1) * (L + 1)];        // C(c, e) z_m^(c-e)
  const int ni = d.ni(), nj = d.nj(), nk = d.nk(), g = d.g;
  const int kb = blockIdx.y * kc, ke = min(kb + kc, nk);
  const int m = ke - kb, np = m / 2;
  const double half_h = 0.5 * hz;
  for (int t = threadIdx.x; t < np; t += blockDim.x) {
    const double u = (double)(m - 1 - 2 * t) * half_h;   // z of plane ke-1-t minus z_m
    double pw = 1.0;
#pragma unroll
    for (int c = 0; c <= L; c++) {
      U[t * (L + 1) + c] = pw;
      pw *= u;
    }
  }
  for (int q0 = threadIdx.x; q0 < (L + 1) * (L + 1); q0 += blockDim.x) {
    const int c = q0 / (L + 1), e = q0 % (L + 1);
    double w = 0.0;
    if (e <= c) {
      const double zm = fma((double)(kb + 1 + ke), half_h, z0);   // planes kb..ke-1 sit at z0 + (k+1) hz
      double binom = 1.0;
      for (int q = 1; q <= e; q++) binom = binom * (double)(c - e + q) / (double)q;
      double zp = 1.0;
      for (int q = 0; q < c - e; q++) zp *= zm;
      w = binom * zp;
    }
    Wsh[q0] = w;
  }
  __syncthreads();
  const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (col >= (long long)ni * nj) return;
  const int i = (int)(col % ni), j = (int)(col / ni);
  double mu[L + 1];
#pragma unroll
  for (int c = 0; c <= L; c++) mu[c] = 0.0;
  const long long sz = d.sz();
  const double* lo = rho + d.at(i + g, j + g, kb + g);
  const double* hi = rho + d.at(i + g, j + g, ke - 1 + g);
  for (int t = 0; t < np; t++, lo += sz, hi -= sz) {
    const double rl = *lo, rh = *hi;
    const double sum = rh + rl, dif = rh - rl;
    const double* up = U + t * (L + 1);
    mu[0] += sum;
#pragma unroll
    for (int c = 1; c <= L; c++) mu[c] = fma((c & 1) ? dif : sum, up[c], mu[c]);
  }
  if (m & 1) mu[0] += *lo;   // the middle plane (u = 0)
  const long long plane = (long long)ni * nj;
  double* out = colmom + (long long)blockIdx.y * (L + 1) * plane + col;
#pragma unroll
  for (int c = 0; c <= L; c++) {
    double v = 0.0;
#pragma unroll
    for (int e = 0; e <= c; e++) v = fma(Wsh[c * (L + 1) + e], mu[e], v);
    out[c * plane] = v;
  }
}

__device__ __forceinline__ int pair_index(int b, int c, int L) {
  // pairs (b, c) with b + c <= L ordered by b, then c
  return b * (L + 1) - b * (b - 1) / 2 + c;
}

// Pass 2: y-moments of the column sums over one y-chunk of 32 rows,
// Y_bc(i) = sum_j y_j^b S_c(i, j), summed over the z-chunks.  Block = 8 warps
// over (x tile of 32, power c, y-chunk); lanes over x (coalesced), warps over
// the chunk's rows; the 8 warp partials are added in warp order.
constexpr int MP_JT = 32;   // rows per y-chunk

template <int L>
__global__ void __launch_bounds__(256)
    k_mp_ycols(Dims d, double y0, double hy, int nchunk, const double* __restrict__ colmom,
               double* __restrict__ ypart) {
  __shared__ double red[8][L + 1][32];
  const int ni = d.ni(), nj = d.nj();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int c = blockIdx.y;
  const int nb = L - c + 1;
  const int jb = blockIdx.z * MP_JT, je = min(jb + MP_JT, nj);
  const long long plane = (long long)ni * nj;
  double acc[L + 1];
#pragma unroll
  for (int b = 0; b <= L; b++) acc[b] = 0.0;
  if (i < ni) {
    for (int q = 0; q < nchunk; q++) {
      const double* src = colmom + ((long long)q * (L + 1) + c) * plane + i;
      for (int j = jb + w; j < je; j += 8) {
        const double y = fma((double)(j + 1), hy, y0);
        double pw = src[(long long)j * ni];
#pragma unroll
        for (int b = 0; b <= L; b++) {
          if (b < nb) acc[b] += pw;
          pw *= y;
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b <= L; b++) red[w][b][lane] = acc[b];
  __syncthreads();
  const int P2 = (L + 1) * (L + 2) / 2;
  for (int t = threadIdx.x; t < nb * 32; t += blockDim.x) {
    const int b = t >> 5, l = t & 31;
    double sum = 0.0;
#pragma unroll
    for (int ww = 0; ww < 8; ww++) sum += red[ww][b][l];
    const int ii = blockIdx.x * 32 + l;
    if (ii < ni) ypart[((long long)blockIdx.z * P2 + pair_index(b, c, L)) * ni + ii] = sum;
  }
}

// Pass 3: x-moments M_abc = dV sum_i x_i^a Y_bc(i), Y summed over the y-chunks:
// one block per monomial slot (threads over x, then a block sum), so that the
// FP64 work is spread over the SMs instead of one SM's narrow FP64 pipe.
__global__ void __launch_bounds__(256)
    k_mp_xmom(Dims d, double x0, double hx, double dV, int L, int njc, const double* __restrict__ ypart,
              double* __restrict__ M) {
  const int W = L + 1;
  const int P2 = W * (W + 1) / 2;
  const int ni = d.ni();
  const int t = blockIdx.x;
  const int c = t % W, b = (t / W) % W, a = t / (W * W);
  if (a + b + c > L) {
    if (threadIdx.x == 0) M[t] = 0.0;
    return;   // uniform over the block
  }
  const int pi = pair_index(b, c, L);
  double acc = 0.0;
  for (int i = threadIdx.x; i < ni; i += blockDim.x) {
    double y = 0.0;
    for (int jc = 0; jc < njc; jc++) y += ypart[((long long)jc * P2 + pi) * ni + i];
    const double x = fma((double)(i + 1), hx, x0);
    double xa = 1.0;
    for (int e = 0; e < a; e++) xa *= x;
    acc = fma(y, xa, acc);
  }
  __shared__ double red[32];
  double v[1] = {acc};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) M[t] = v[0] * dV;
}

// q_lm = sum over the monomials of R_lm's coefficient times M_abc (sparse table).
__global__ void __launch_bounds__(256)
    k_mp_q(int L, const double* __restrict__ M, const int* __restrict__ off, const int* __restrict__ mono,
           const double* __restrict__ val, double* __restrict__ q) {
  const int W = L + 1;
  for (int lm = threadIdx.x; lm < W * W; lm += blockDim.x) {
    double acc = 0.0;
    for (int t = off[lm]; t < off[lm + 1]; t++) acc = fma(val[t], M[mono[t]], acc);
    q[lm] = acc;
  }
}

// ------------------------------------------------------------------ boundary values
// F(u, v, w) = sum_{a+b+c <= L} C_abc u^a v^b w^c by nested Horner (w, then v,
// then u); C dense over (L+1)^3 slots.
__device__ __forceinline__ double eval_boundary_poly(double u, double v, double w, int L,
                                                     const double* __restrict__ C) {
  const int W = L + 1;
  double F = 0.0;
  for (int a = L; a >= 0; a--) {
    double Gv = 0.0;
    for (int b = L - a; b >= 0; b--) {
      const double* cb = C + (a * W + b) * W;
      double H = cb[L - a - b];
      for (int c = L - a - b - 1; c >= 0; c--) H = fma(H, w, cb[c]);
      Gv = b == L - a ? H : fma(Gv, v, H);
    }
    F = a == L ? Gv : fma(F, u, Gv);
  }
  return F;
}

__global__ void __launch_bounds__(256)
    k_mp_faces(Dims d, double x0, double y0, double z0, double hx, double hy, double hz, int L,
               double G, const double* __restrict__ q, const int* __restrict__ toff,
               const int* __restrict__ tlm, const double* __restrict__ tval, double* __restrict__ phi) {
  // the boundary polynomial C_abc = sum over lm of q_lm times R_lm's coefficient
  // of x^a y^b z^c (transposed table; zero where a+b+c > L), per block
  extern __shared__ double poly[];
  const int W = L + 1;
  for (int t = threadIdx.x; t < W * W * W; t += blockDim.x) {
    double acc = 0.0;
    for (int e = toff[t]; e < toff[t + 1]; e++) acc = fma(tval[e], q[tlm[e]], acc);
    poly[t] = acc;
  }
  __syncthreads();
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
  const double ir = rsqrt(fma(x, x, fma(y, y, z * z)));
  const double t = ir * ir;
  phi[d.at(i, j, k)] = -G * ir * eval_boundary_poly(x * t, y * t, z * t, L, poly);
}

// ------------------------------------------------------------------ host launchers
// z-chunks of pass 1: enough columns x chunks for about 1024 threads per SM
static int mp_chunks(const Dims& d) {
  const long long cols = (long long)d.ni() * d.nj();
  long long nc = (device_sm_count() * 1024LL + cols - 1) / cols;
  nc = std::max(nc, (long long)((d.nk() + MP_KC_MAX - 1) / MP_KC_MAX));
  return (int)std::max(1LL, std::min(nc, (long long)d.nk()));
}

cudaError_t cart_multipole_alloc(const Dims& d, int lmax, const MultipoleTables& t,
                                 CartMultipoleDev* m) {
  const int W = lmax + 1;
  m->lmax = lmax;
  m->nchunk = mp_chunks(d);
  size_t ncol = (size_t)m->nchunk * W * d.ni() * d.nj();
  size_t ny = (size_t)((d.nj() + MP_JT - 1) / MP_JT) * d.ni() * W * (W + 1) / 2;
  cudaError_t e;
  if ((e = cudaMalloc(&m->colmom, ncol * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->ymom, ny * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->mom, (size_t)W * W * W * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->q, (size_t)W * W * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->off, t.off.size() * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->mono, std::max<size_t>(1, t.mono.size()) * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->val, std::max<size_t>(1, t.val.size()) * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->toff, t.toff.size() * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->tlm, std::max<size_t>(1, t.tlm.size()) * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m->tval, std::max<size_t>(1, t.tval.size()) * sizeof(double))) != cudaSuccess) return e;
  m->bytes = (ncol + ny + W * W * W + W * W + 2 * t.val.size()) * sizeof(double) +
             (t.off.size() + t.toff.size() + 2 * t.mono.size()) * sizeof(int);
  if ((e = cudaMemcpy(m->off, t.off.data(), t.off.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(m->toff, t.toff.data(), t.toff.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if (!t.mono.empty()) {
    if ((e = cudaMemcpy(m->mono, t.mono.data(), t.mono.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(m->val, t.val.data(), t.val.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(m->tlm, t.tlm.data(), t.tlm.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(m->tval, t.tval.data(), t.tval.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

size_t cart_multipole_bytes(const Dims& d, int lmax) {
  const size_t W = lmax + 1;
  // table entries: at most (l+1)(l+2)/2 monomials for each of the 2l+1 R_lm of degree l
  size_t ent = 0;
  for (size_t l = 0; l < W; l++) ent += (2 * l + 1) * (l + 1) * (l + 2) / 2;
  return ((size_t)mp_chunks(d) * W * d.ni() * d.nj() +
          (size_t)((d.nj() + MP_JT - 1) / MP_JT) * d.ni() * W * (W + 1) / 2 + W * W * W + W * W + 4096) *
             sizeof(double) +
         ent * 2 * (sizeof(double) + sizeof(int)) + (W * W + W * W * W + 2) * sizeof(int);
}

void cart_multipole_free(CartMultipoleDev* m) {
  cudaFree(m->colmom);
  cudaFree(m->ymom);
  cudaFree(m->mom);
  cudaFree(m->q);
  cudaFree(m->off);
  cudaFree(m->mono);
  cudaFree(m->val);
  cudaFree(m->toff);
  cudaFree(m->tlm);
  cudaFree(m->tval);
  *m = CartMultipoleDev();
}

template <int L>
static void passes12(const Dims& d, double y0, double hy, double z0, double hz, int nchunk_alloc,
                     const double* rho, double* colmom, double* ypart, cudaStream_t s) {
  const long long cols = (long long)d.ni() * d.nj();
  const int kc = (d.nk() + nchunk_alloc - 1) / nchunk_alloc;
  const int nchunk = (d.nk() + kc - 1) / kc;
  const dim3 g1((unsigned)((cols + 255) / 256), (unsigned)nchunk);
  k_mp_cols<L><<<g1, 256, 0, s>>>(d, z0, hz, kc, rho, colmom);
  const dim3 g2((unsigned)((d.ni() + 31) / 32), L + 1, (unsigned)((d.nj() + MP_JT - 1) / MP_JT));
  k_mp_ycols<L><<<g2, 256, 0, s>>>(d, y0, hy, nchunk, colmom, ypart);
}

// Moments about the origin in three separable passes (z, then y, then x),
// then the map to q_lm.  Launches: 4.
cudaError_t launch_cart_moments(const Dims& d, const double lo[3], const double h[3],
                                const double origin[3], const double* rho, CartMultipoleDev* m,
                                cudaStream_t s) {
  const int L = m->lmax;
  if (L < 0 || L > MAXL) return cudaErrorInvalidValue;
  if ((d.nk() + m->nchunk - 1) / m->nchunk > MP_KC_MAX) return cudaErrorInvalidValue;
  const double dV = h[0] * h[1] * h[2];
  const double y0 = lo[1] - origin[1], z0 = lo[2] - origin[2];
#define PS_MP_CASE(LL) \
  case LL: passes12<LL>(d, y0, h[1], z0, h[2], m->nchunk, rho, m->colmom, m->ymom, s); break;
  switch (L) {
    PS_MP_CASE(0) PS_MP_CASE(1) PS_MP_CASE(2) PS_MP_CASE(3) PS_MP_CASE(4) PS_MP_CASE(5)
    PS_MP_CASE(6) PS_MP_CASE(7) PS_MP_CASE(8) PS_MP_CASE(9) PS_MP_CASE(10) PS_MP_CASE(11)
    PS_MP_CASE(12) PS_MP_CASE(13) PS_MP_CASE(14) PS_MP_CASE(15)
    default: passes12<16>(d, y0, h[1], z0, h[2], m->nchunk, rho, m->colmom, m->ymom, s); break;
  }
#undef PS_MP_CASE
  const int W = L + 1;
  const int njc = (d.nj() + MP_JT - 1) / MP_JT;
  k_mp_xmom<<<W * W * W, 256, 0, s>>>(d, lo[0] - origin[0], h[0], dV, L, njc, m->ymom, m->mom);
  k_mp_q<<<1, 256, 0, s>>>(L, m->mom, m->off, m->mono, m->val, m->q);
  return cudaGetLastError();
}

cudaError_t launch_cart_faces(const Dims& d, const double lo[3], const double h[3],
                              const double origin[3], double G, const double* q,
                              const CartMultipoleDev* m, double* phi, cudaStream_t s) {
  const long long total = 2LL * d.g * ((long long)d.ex * d.ey + (long long)d.ex * d.nk() +
                                       (long long)d.nj() * d.nk());
  const int thr = 256;
  const long long blocks = (total + thr - 1) / thr;
  const size_t W = m->lmax + 1;
  k_mp_faces<<<(unsigned)blocks, thr, W * W * W * sizeof(double), s>>>(
      d, lo[0] - origin[0], lo[1] - origin[1], lo[2] - origin[2], h[0], h[1], h[2], m->lmax, G, q, m->toff,
      m->tlm, m->tval, phi);
  return cudaGetLastError();
}

}  // namespace ps
