// Multipole open boundary (Sec. 2.2): moments (Eq. outer_multipole) and the
// truncated outer expansion (Eq. outer_expansion) on boundary nodes.
#pragma once
#include <vector>

#include "ps_common.cuh"

namespace ps {

// Regular solid harmonics in Schmidt (Racah) normalisation,
//   R_lm(x) = sqrt(4 pi / (2l+1)) r^l Y_lm(x),
// so that q_lm = sum rho dV R_lm(x') and Phi(x) = -G sum q_lm R_lm(x) / r^(2l+1).
// Host tables shared by the Cartesian and spherical kernels.
struct MultipoleTables {
  int lmax = -1;
  // Cartesian: R_lm as a sparse polynomial sum_k val[k] x^a y^b z^c with
  // mono[k] = (a*(L+1) + b)*(L+1) + c, terms of (l,m) in [off[lm], off[lm+1]).
  std::vector<int> off, mono;
  std::vector<double> val;
  // the transpose: per monomial slot t = (a*(L+1) + b)*(L+1) + c, the pairs
  // (lm, val) of the R_lm that contain x^a y^b z^c, in [toff[t], toff[t+1])
  std::vector<int> toff, tlm;
  std::vector<double> tval;
  // recurrence constants for direct evaluation: rec_a[l*(L+1)+m] = (2l-1)/(l-m),
  // rec_b = (l+m-1)/(l-m) for l >= m+2; nrm[l*(L+1)+m] = sqrt(2 (l-m)!/(l+m)!) (m>0), 1 (m=0);
  // dfac[m] = (2m-1)!!
  std::vector<double> rec_a, rec_b, nrm, dfac;
};

void build_multipole_tables(int lmax, MultipoleTables* t);

struct CartMultipoleDev {
  int lmax = -1;
  int nchunk = 1;              // z-chunks of the column pass
  double* colmom = nullptr;    // [nchunk][L+1][nj][ni] column z-moments
  double* ymom = nullptr;      // [y-chunks][(L+1)(L+2)/2][ni] y-moments of the column sums
  double* mom = nullptr;       // [(L+1)^3] monomial moments M_abc (zero where a+b+c > L)
  double* q = nullptr;         // [(L+1)^2]
  int* off = nullptr;
  int* mono = nullptr;
  double* val = nullptr;
  int* toff = nullptr;         // transposed table (see MultipoleTables)
  int* tlm = nullptr;
  double* tval = nullptr;
  size_t bytes = 0;
};

cudaError_t cart_multipole_alloc(const Dims& d, int lmax, const MultipoleTables& t,
                                 CartMultipoleDev* m);
void cart_multipole_free(CartMultipoleDev* m);
// device bytes cart_multipole_alloc takes for a grid (admission estimates)
size_t cart_multipole_bytes(const Dims& d, int lmax);

// q (device) <- moments of rho over interior nodes about origin (weights h^3).
cudaError_t launch_cart_moments(const Dims& d, const double lo[3], const double h[3],
                                const double origin[3], const double* rho, CartMultipoleDev* m,
                                cudaStream_t s);
// phi <- -G sum q R / r^(2l+1) on every non-interior node.
cudaError_t launch_cart_faces(const Dims& d, const double lo[3], const double h[3],
                              const double origin[3], double G, const double* q,
                              const CartMultipoleDev* m, double* phi, cudaStream_t s);

}  // namespace ps
