// Device code shared by the per-solve kernels (cart_kernels.cu) and the
// batched kernels (batch.cu): the Gauss-Seidel value of a node, the
// coarsest-level CG of one thread block, and the residual-norm finisher.
#pragma once
#include "ps_common.cuh"

namespace ps {

// ------------------------------------------------------------------ stencil core
// phi_GS without the diagonal: sum of weighted neighbours plus fs.
template <int G, bool ISO, typename T, typename C>
__device__ __forceinline__ C gs_value(const T* __restrict__ phi, long long p, long long sy,
                                      long long sz, const Coef<C>& cf, C fs) {
  using S = St<T>;
  C ax = S::ld(phi + p + 1) + S::ld(phi + p - 1);
  C v;
  if constexpr (ISO && G == 1 && sizeof(C) == 8) {
    // FP64 7-point on equal spacings: the order of the diagonal colour pass
    // (k_sweep_diag), (E + W) + (S + D) + (N + U), so that residuals after a
    // sweep repeat its arithmetic exactly
    const C sd = S::ld(phi + p - sy) + S::ld(phi + p - sz);
    const C nu = S::ld(phi + p + sy) + S::ld(phi + p + sz);
    return fma((ax + sd) + nu, cf.c1[0], fs);
  }
  if constexpr (ISO && G == 2 && sizeof(C) == 8) {
    // FP64 13-point on equal spacings: the order of the diagonal colour pass
    // (k_sweep_diag13), (E + W) + (S + U) + (N + D) at distance 1, then the
    // same at distance 2
    const C su1 = S::ld(phi + p - sy) + S::ld(phi + p + sz);
    const C nd1 = S::ld(phi + p + sy) + S::ld(phi + p - sz);
    const C v1 = fma((ax + su1) + nd1, cf.c1[0], fs);
    const C ew2 = S::ld(phi + p + 2) + S::ld(phi + p - 2);
    const C su2 = S::ld(phi + p - 2 * sy) + S::ld(phi + p + 2 * sz);
    const C nd2 = S::ld(phi + p + 2 * sy) + S::ld(phi + p - 2 * sz);
    return fma((ew2 + su2) + nd2, cf.c2[0], v1);
  }
  C ay = S::ld(phi + p + sy) + S::ld(phi + p - sy);
  C az = S::ld(phi + p + sz) + S::ld(phi + p - sz);
  if (ISO) {
    v = fma((ax + ay) + az, cf.c1[0], fs);
  } else {
    v = fma(ax, cf.c1[0], fma(ay, cf.c1[1], fma(az, cf.c1[2], fs)));
  }
  if (G == 2) {
    C bx = S::ld(phi + p + 2) + S::ld(phi + p - 2);
    C by = S::ld(phi + p + 2 * sy) + S::ld(phi + p - 2 * sy);
    C bz = S::ld(phi + p + 2 * sz) + S::ld(phi + p - 2 * sz);
    if (ISO) {
      v = fma((bx + by) + bz, cf.c2[0], v);
    } else {
      v = fma(bx, cf.c2[0], fma(by, cf.c2[1], fma(bz, cf.c2[2], v)));
    }
  }
  return v;
}

// Set the enclosing graph's while-condition (chunk > 0 marks a graph body):
// continue while not done and below the iteration budget of this step, so
// every graph launch ends after a bounded number of iterations.
__device__ __forceinline__ void set_loop(const DevState* st, unsigned long long cond, int chunk) {
  if (chunk > 0) {
    const unsigned int more = (st->done == DONE_NO && st->iter < st->chunk_end) ? 1u : 0u;
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond, more);
  }
}

// Sum a residual pass's per-block partials {sum delta^2, max |delta|} in block
// order, record the norm in the state and decide convergence (one block).
// mode: 0 = reference norm, 1 = initial residual, 2 = iteration check, 3 =
// iteration check that calls only a non-finite norm divergence (SOR on graded
// spherical grids: its non-normal iteration grows the residual a
// hundred-to-thousandfold before it converges), 4 = initial residual whose
// pass returned early on a zero guess (st->guess_nonzero == 0): the residual
// is then the reference vector, and its norm and max are those of mode 0.
__device__ __forceinline__ void finish_norm_block(const double* __restrict__ partials, int nblocks,
                                                  double dscale, int mode, DevState* __restrict__ st,
                                                  unsigned long long cond, int chunk) {
  __shared__ double red[64];
  const bool from_ref = mode == 4 && st->guess_nonzero == 0;
  if (mode == 4) mode = 1;
  double s = 0.0, m = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    s += partials[2 * b];
    m = fmax(m, partials[2 * b + 1]);
  }
  double a[1] = {s};
  block_sum<1>(a, red);
  // max over the block
  m = warp_max(m);
  __shared__ double mx[32];
  if ((threadIdx.x & 31) == 0) mx[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x + 31) / 32; w++) m = fmax(m, mx[w]);
  m = fmax(m, mx[0]);
  const double S = a[0];
  const double rr = from_ref ? st->rr : dscale * dscale * S;
  if (from_ref) m = st->amax;
  if (mode == 0) {
    st->rr = rr;
    double ref = sqrt(rr);
    st->ref = ref > 0.0 ? ref : 1.0;
    st->amax = m;
    st->scale_next = m > 0.0 ? exp2(-rint(log2(m))) : 1.0;
    return;
  }
  if (st->done && mode >= 2) {
    set_loop(st, cond, chunk);
    return;
  }
  if (st->fault) {
    st->done = DONE_FAULT;
    set_loop(st, cond, chunk);
    return;
  }
  st->rr = rr;
  st->amax = m;
  const double rel = sqrt(rr) / st->ref;
  st->rel = rel;
  // IR: the scale of the next stored inner right-hand side (power of two)
  st->scale_cur = st->scale_next;
  st->scale_next = m > 0.0 ? exp2(-rint(log2(m))) : 1.0;
  if (mode == 1) {
    st->iter = 0;
    st->rel0 = rel;
    st->done = rel <= st->tol ? DONE_CONVERGED : (st->max_iter <= 0 ? DONE_MAXITER : DONE_NO);
    if (!isfinite(rel)) st->done = DONE_DIVERGED;
    return;
  }
  st->iter += 1;
  if (!isfinite(rel) || (mode == 2 && rel > 1e3 * fmax(st->rel0, 1.0))) st->done = DONE_DIVERGED;
  else if (rel <= st->tol) st->done = DONE_CONVERGED;
  else if (st->iter >= st->max_iter) st->done = DONE_MAXITER;
  set_loop(st, cond, chunk);
}

// ------------------------------------------------------------------ coarsest-level CG
// One CTA solves -A e = d * fs (zero boundary, e0 = 0) by CG (Sec. 2.1.3: the
// coarsest level is solved with CG) until ||r|| <= tol ||r0|| or max_iter
// iterations.  Each thread owns up to PPT unknowns and keeps their x, r, q in
// registers; only the search direction p lives in shared memory (on the full
// ghosted layout, zero boundary), because the stencil reads neighbours.
// GB300's FP64 pipe is narrow, so the FP64 work that is not per unknown is done
// once: each dot product is one per-thread partial in shared memory summed by
// warp 0 (a strided loop, then one shuffle tree), and thread 0 alone forms
// alpha, beta and the convergence test and hands them out through shared memory.
// About 100 threads with several unknowns each keep the pipe busy with
// independent work while the block's barriers stay cheap.
// p: shared memory holding the whole ghosted level (d.size() doubles).
template <int G, bool ISO, typename TF, typename TE, int PPT, int MAXT>
__device__ __forceinline__ void coarse_cg_block(const Dims& d, const Coef<double>& cf,
                                                const TF* __restrict__ fs, TE* __restrict__ e,
                                                double tol, int max_iter, DevState* __restrict__ st,
                                                double* p) {
  __shared__ double part[MAXT];
  __shared__ double scal[2];   // alpha / beta handed out by thread 0
  __shared__ int stop;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  const int ni = d.ni(), nj = d.nj(), nk = d.nk();
  const int nint = ni * nj * nk;
  const long long n = d.size();
  const long long sy = d.sy(), sz = d.sz();
  // block sum of v into lane values of warp 0 (valid in thread 0)
  auto block_sum0 = [&](double v) -> double {
    part[tid] = v;
    __syncthreads();
    double t = 0.0;
    if (tid < 32) {
      for (int i = lane; i < nthr; i += 32) t += part[i];
      t = warp_sum(t);
    }
    return t;
  };
  for (long long u = tid; u < n; u += nthr) p[u] = 0.0;
  long long c[PPT];
  double x[PPT], r[PPT], q[PPT];
  bool own[PPT];
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const int u = tid + k * nthr;
    own[k] = u < nint;
    const int uu = own[k] ? u : 0;
    const int i = uu % ni, t = uu / ni;
    c[k] = d.at(i + G, t % nj + G, t / nj + G);
    x[k] = 0.0;
    r[k] = 0.0;
    q[k] = 0.0;
  }
  __syncthreads();
  double loc = 0.0;
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    if (own[k]) {
      const double b = cf.d * (double)St<TF>::ld(fs + c[k]);
      r[k] = b;
      p[c[k]] = b;
      loc = fma(b, b, loc);
    }
  }
  // thread 0 keeps rr, ref and the iteration count
  double rr = block_sum0(loc);
  double ref = 0.0;
  int it = 0;
  if (tid == 0) {
    ref = sqrt(rr);
    stop = !(ref > 0.0) || max_iter <= 0;
  }
  __syncthreads();
  while (!stop) {
    loc = 0.0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      if (own[k]) {
        const double pc = p[c[k]];
        q[k] = cf.d * (pc - gs_value<G, ISO>(p, c[k], sy, sz, cf, 0.0));
        loc = fma(pc, q[k], loc);
      }
    }
    const double pq = block_sum0(loc);
    if (tid == 0) scal[0] = rr / pq;
    __syncthreads();
    const double alpha = scal[0];
    loc = 0.0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      if (own[k]) {
        x[k] = fma(alpha, p[c[k]], x[k]);
        r[k] = fma(-alpha, q[k], r[k]);
        loc = fma(r[k], r[k], loc);
      }
    }
    const double rrn = block_sum0(loc);
    if (tid == 0) {
      it++;
      stop = sqrt(rrn) <= tol * ref || it >= max_iter;
      scal[1] = rrn / rr;
      rr = rrn;
    }
    __syncthreads();   // every thread is past its stencil reads of p
    if (stop) break;
    const double beta = scal[1];
#pragma unroll
    for (int k = 0; k < PPT; k++)
      if (own[k]) p[c[k]] = fma(beta, p[c[k]], r[k]);
    __syncthreads();   // p complete
  }
#pragma unroll
  for (int k = 0; k < PPT; k++)
    if (own[k]) St<TE>::st(e + c[k], (typename St<TE>::C)x[k]);
  if (tid == 0 && st != nullptr) {
    st->coarse_iter_last = it;
    st->coarse_iter_total += it;
  }
}

}  // namespace ps
