// Host drivers and C ABI of the GB300 Poisson library (include/poisson.h).
//
// poisson_create builds the level list and allocates the device hierarchy;
// poisson_solve runs, on one stream:
//   multipole moments + boundary values (Sec. 2.2)            [t_mp]
//   f = 4 pi G rho scaled to the Gauss-Seidel form
//   reference and initial residual norms
//   the iteration: SOR steps (Sec. 2.1.1), CG or BiCGSTAB iterations
//   (Sec. 2.1.2), V(nu1,nu2) cycles (Sec. 2.1.3) or FP64 iterative refinement
//   around FP32/BF16 inner V-cycles or FP32 inner BiCGSTAB       [t_iter]
// Convergence is decided on the device; the host reads the small state once per
// V-cycle / refinement step, or once per chunk of Krylov/SOR iterations (the
// kernels of an iteration body skip their work once the state says done).
#include <atomic>
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "cart_kernels.cuh"
#include "tiled_kernels.cuh"
#include "batch.cuh"
#include "multipole.cuh"
#include "spherical.cuh"
#include "compact.cuh"

namespace ps {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 152;
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

static size_t dt_size(int dt) { return dt == DT_F64 ? 8 : dt == DT_F32 ? 4 : 2; }

struct Level {
  Dims d{};
  double h[3] = {0, 0, 0};
  int dt = DT_F64;       // storage of phi and fs
  int dt_tmp = DT_F64;   // storage of the delta buffer fed to the restriction
  void* phi = nullptr;
  void* phib = nullptr;  // second potential buffer of the out-of-place (fused) sweeps
  void* fs = nullptr;
  void* tmp = nullptr;
  bool own_phi = true, own_phib = true, own_fs = true;
};

struct Hier {
  bool built = false;
  std::vector<Level> lv;
  size_t bytes = 0;
};

static const int KRYLOV_CHUNK = 16;
// Coarsest-level CG tolerance: Sec. 2.1.3 -- a relative accuracy of about the
// V-cycle convergence factor (~0.075 here) keeps the asymptotic rate; 1e-2 stays
// an order of magnitude below it.
static const double COARSE_TOL = 1e-2;

}  // namespace ps

using namespace ps;

// Kernel classes of the opt-in profiler.
enum ProfClass {
  PC_SWEEP0 = 0, PC_DELTA0, PC_RESTRICT0, PC_PROLONG0, PC_NORM0, PC_COARSE, PC_MOMENTS, PC_FACES,
  PC_SWEEP_C, PC_CORRECT0, PC_KRYLOV, PC_RBSWEEP0, PC_RBSWEEP_C, PC_RESTRICT_FUSED0, PC_RHS0, PC_COUNT
};
static const char* kProfNames[PC_COUNT] = {
  "sweep_colour_finest", "residual_finest", "restrict_finest", "prolong_finest", "norm_finest",
  "coarse_cg", "multipole_moments", "multipole_boundary", "sweep_colour_coarse", "ir_correct",
  "krylov_vector", "sweep_fused_finest", "sweep_fused_coarse", "resid_restrict_finest", "rhs_finest"};

// One iteration of a solve, enqueued on a stream; cond/chunk are set when it is
// being captured into a loop graph.
using Body = std::function<cudaError_t(unsigned long long, int, cudaStream_t)>;

// The solve in flight on a handle (begin .. end).
struct Active {
  bool on = false;
  ps_solve_opts o{};
  double tol = 0.0;
  const double* rho = nullptr;
  double* phi_user = nullptr;
  cudaStream_t caller = nullptr;
  std::string key;
  Body body;
  int chunk = 32, plain_chunk = 1;
  bool plain_steps = false;
  bool count_replacements = false;   // inner_cycles reports FP32 BiCGSTAB residual replacements
  int sweep_tile = 0;                 // tile variant of the fused FP32/BF16 sweeps (0 = default)
  int restrict_tile = 0;              // tile variant of the fused FP32/BF16 residual + restriction
  long long body_kernels = 0;
  int inner_per_iter = 0;
  // enqueued by every step before the iterations / after them (may be empty)
  std::function<cudaError_t(cudaStream_t)> prologue, epilogue;
};

// A captured iteration body inside a CUDA-graph while loop.
struct LoopGraph {
  cudaGraphExec_t exec = nullptr;
  long long body_kernels = 0;
};

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
  double bytes, ops;
  int fp64;
  int variant;
};

// Per-kernel-class totals of timed launches.
struct ProfAcc {
  long long n = 0;
  double ms = 0.0, bytes = 0.0, ops = 0.0;
  int fp64 = 0;
  int variant = 0;
};

// A captured iteration body with CUDA-event record nodes around its hot
// kernels (a plain graph: event nodes cannot sit inside conditional bodies).
struct ProfGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<ProfRec> slots;
  long long body_kernels = 0;
};

struct ps_ctx {
  ps_grid grid{};
  int order = 2;
  ps_bc bc{};
  int lmax = 0;
  bool sph = false;
  cudaStream_t stream = nullptr;
  DevState* st = nullptr;    // device
  DevState* hst = nullptr;   // pinned host mirror
  double* partials = nullptr;
  int npart = 0;
  // Cartesian
  Dims d0{};                // finest level, library layout (pitched rows)
  Dims du{};                // finest level as the caller stores rho and phi (dense)
  double h0[3] = {0, 0, 0};
  int nlev = 0;
  std::vector<Dims> dims;
  std::vector<std::array<double, 3>> hs;
  Hier h64, hmx[2];
  double* fs64 = nullptr;
  double *cg_r = nullptr, *cg_p = nullptr, *cg_q = nullptr, *cg_z = nullptr;
  MultipoleTables mpt;
  CartMultipoleDev mp;
  // spherical
  SphDims sd{};
  SphTables stab;
  void* sv[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int sv_dt = -1;
  double* sz = nullptr;   // BiCGSTAB group-wise increments of the iterate (FP64)
  double* sph_w = nullptr;   // spherical SOR weights, two buffers of Ntheta * Nr
  double* sph_g = nullptr;   // spherical SOR: scaled right-hand side -f / a_c (field layout)
  ps_tuning tun[3] = {};     // tuned multigrid settings per precision (poisson_set_tuning)
  int has_tun[3] = {0, 0, 0};
  // Cartesian SOR: weights of the Chebyshev sequence, one per colour pass
  double* sor_wtab = nullptr;
  int sor_wlen = 0;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  size_t bytes = 0;
  // profiler
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<ProfRec>* cap_slots = nullptr;   // non-null while capturing a profiling graph
  std::map<std::string, ProfGraph> pgraphs;
  ProfAcc acc[PC_COUNT];
  std::vector<cudaEvent_t> ev_pool;
  int prof_open = -1;
  long long nlaunch = 0;   // kernels launched by the current solve
  // captured loop bodies (keyed by method and parameters) and their capture stream
  std::map<std::string, LoopGraph> graphs;
  cudaStream_t cap = nullptr;
  double* phi0 = nullptr;  // internal finest-level potential (Cartesian) / unknowns (spherical)
  Active act;
  bool in_batch = false;           // the handle's hierarchy is advanced by a batch
  DevState* st_active = nullptr;   // the state the loop gate reads (= st)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace {

ps_status fail(ps_status s, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

// Arithmetic instructions per fine node of the grid-transfer kernels (FMA = 1).
// Full weighting: per coarse node two carried plane sums of 8 (three row sums of
// an add and an FMA, then an add and an FMA), the z-triple (add, FMA) and the
// scale: 19 per 8 fine nodes.  Trilinear prolongation: per coarse cell one face
// (4 midpoints of an add and a multiply), 4 z-midpoints and 8 accumulations:
// 24 per 8 fine nodes.
constexpr double kRestrictOps = 19.0 / 8.0;
// Full weighting of a residual that is zero on the black nodes: a carried half
// sum of the odd-offset plane (3 adds), the even-offset plane (2 adds, 1 FMA),
// the z-triple (2 adds) and the scale: 9 per 8 fine nodes.
constexpr double kRestrictRedOps = 9.0 / 8.0;
constexpr double kProlongOps = 3.0;

// Profiler: begin/end pair around one launch on stream s.
void prof_begin(ps_ctx* h, int cls, double bytes, double ops, int fp64, cudaStream_t s, int variant = 0) {
  std::vector<ProfRec>& sink = h->cap_slots ? *h->cap_slots : h->recs;
  if (!h->prof || sink.size() >= 16384) return;
  ProfRec r;
  r.cls = cls;
  r.bytes = bytes;
  r.ops = ops;
  r.fp64 = fp64;
  r.variant = variant;
  for (cudaEvent_t* e : {&r.a, &r.b}) {
    if (!h->ev_pool.empty()) {
      *e = h->ev_pool.back();
      h->ev_pool.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      return;
    }
  }
  // inside a stream capture only an external record becomes an event-record node
  if (h->cap_slots) cudaEventRecordWithFlags(r.a, s, cudaEventRecordExternal);
  else cudaEventRecord(r.a, s);
  sink.push_back(r);
  h->prof_open = (int)sink.size() - 1;
}
void prof_end(ps_ctx* h, cudaStream_t s) {
  if (h->prof_open < 0) return;
  std::vector<ProfRec>& sink = h->cap_slots ? *h->cap_slots : h->recs;
  if (h->cap_slots) cudaEventRecordWithFlags(sink[h->prof_open].b, s, cudaEventRecordExternal);
  else cudaEventRecord(sink[h->prof_open].b, s);
  h->prof_open = -1;
}

#define TRY(expr)                                                                      \
  do {                                                                                 \
    cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess) {                                                           \
      return fail(_e == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA,          \
                  "%s:%d: %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(_e)); \
    }                                                                                  \
  } while (0)

bool levels_for(const int n[3], std::vector<std::array<int, 3>>* out) {
  out->clear();
  std::array<int, 3> cur = {n[0], n[1], n[2]};
  out->push_back(cur);
  while (cur[0] % 2 == 0 && cur[1] % 2 == 0 && cur[2] % 2 == 0 && cur[0] >= 16 && cur[1] >= 16 &&
         cur[2] >= 16) {
    for (int a = 0; a < 3; a++) cur[a] /= 2;
    out->push_back(cur);
  }
  return true;
}

// Library-owned level arrays pad rows to 32 elements; the coarsest level,
// which the single-CTA CG keeps whole in shared memory, stays dense.
Dims level_dims(const std::array<int, 3>& n, int gw, bool coarsest) {
  return make_dims(n[0], n[1], n[2], gw, coarsest ? 1 : 32);
}

// Copy a whole FP64 field between two layouts of the same level.
cudaError_t copy_rows(double* dst, const Dims& dd, const double* src, const Dims& sd, cudaStream_t s) {
  return cudaMemcpy2DAsync(dst, (size_t)dd.px * sizeof(double), src, (size_t)sd.px * sizeof(double),
                           (size_t)sd.ex * sizeof(double), (size_t)sd.ey * sd.ez,
                           cudaMemcpyDeviceToDevice, s);
}

ps_status validate_cart(const ps_grid* g, int order) {
  if (order != 2 && order != 4) return fail(PS_ERR_INVALID_ARG, "stencil_order must be 2 or 4 (got %d)", order);
  for (int a = 0; a < 3; a++) {
    if (g->n[a] < 2) return fail(PS_ERR_INVALID_ARG, "n[%d] = %d: need at least 2 intervals", a, g->n[a]);
    if (g->n[a] > 8192) return fail(PS_ERR_INVALID_ARG, "n[%d] = %d too large", a, g->n[a]);
    if (!(g->hi[a] > g->lo[a]) || !std::isfinite(g->hi[a] - g->lo[a]))
      return fail(PS_ERR_INVALID_ARG, "box axis %d: hi must exceed lo", a);
  }
  return PS_OK;
}

[[maybe_unused]] size_t cart_level_bytes(const Dims& d, int dt, bool tmp) {
  return (size_t)d.size() * dt_size(dt) * (tmp ? 3 : 2);
}

ps_status alloc_zero(void** p, size_t bytes, size_t* acc) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  e = cudaMemset(*p, 0, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) return fail(PS_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
  *acc += bytes;
  return PS_OK;
}

// Build a hierarchy. prec 0 = FP64 (level-0 phi is the caller's array, level-0
// fs the handle's fs64); prec 1/2 = mixed FP32 / BF16 finest inner level.
ps_status build_hier(ps_ctx* h, int prec, Hier* H) {
  if (H->built) return PS_OK;
  H->lv.resize(h->nlev);
  for (int l = 0; l < h->nlev; l++) {
    Level& L = H->lv[l];
    L.d = h->dims[l];
    for (int a = 0; a < 3; a++) L.h[a] = h->hs[l][a];
    if (prec == 0) {
      L.dt = DT_F64;
      L.dt_tmp = DT_F64;
    } else {
      L.dt = (l == 0 && prec == 2) ? DT_BF16 : DT_F32;
      L.dt_tmp = DT_F32;
    }
    const size_t n = (size_t)L.d.size();
    const bool pingpong = h->order == 2 && l + 1 < h->nlev;   // fused sweeps possible
    ps_status s;
    if (prec == 0 && l == 0) {
      L.own_phi = false;
      L.own_fs = false;
      L.fs = h->fs64;
    } else {
      if ((s = alloc_zero(&L.phi, n * dt_size(L.dt), &H->bytes)) != PS_OK) return s;
      if ((s = alloc_zero(&L.fs, n * dt_size(L.dt), &H->bytes)) != PS_OK) return s;
      if (pingpong && L.dt != DT_F64 && (s = alloc_zero(&L.phib, n * dt_size(L.dt), &H->bytes)) != PS_OK) return s;
    }
    if (l + 1 < h->nlev)
      if ((s = alloc_zero(&L.tmp, n * dt_size(L.dt_tmp), &H->bytes)) != PS_OK) return s;
  }
  H->built = true;
  h->bytes += H->bytes;
  return PS_OK;
}

void free_hier(Hier* H) {
  for (auto& L : H->lv) {
    if (L.own_phi) cudaFree(L.phi);
    if (L.own_phib) cudaFree(L.phib);
    if (L.own_fs) cudaFree(L.fs);
    cudaFree(L.tmp);
  }
  H->lv.clear();
  H->built = false;
}

// Algorithmic work of the finest-level passes (per launch), for the profiler.
struct Work {
  double n;       // interior unknowns
  double S, St;   // storage bytes of phi/fs and of the delta buffer
  int G;
  bool fp64;
};
Work work_of(const Level& L, int order) {
  Work w;
  w.n = (double)L.d.ni() * L.d.nj() * L.d.nk();
  w.S = (double)dt_size(L.dt);
  w.St = (double)dt_size(L.dt_tmp);
  w.G = order / 2;
  w.fp64 = L.dt == DT_F64;
  return w;
}

cudaError_t sweep_level(ps_ctx* h, Level& L, int l, double omega, const DevState* st, cudaStream_t s,
                        const double* wtab = nullptr, int wlen = 0, int first_colour = 0) {
  const int ncol = h->order == 2 ? 2 : 3;
  const Work w = work_of(L, h->order);
  cudaError_t e;
  // FP64 passes on equal spacings walk (j, k) diagonals: 5 FP64 instructions
  // per update instead of 6 (13-point: 10 instead of 12)
  const bool diag = L.dt == DT_F64 && L.h[0] == L.h[1] && L.h[1] == L.h[2];
  const double per_update = diag ? 5.0 * w.G : 6.0 * w.G;
  for (int c = first_colour; c < ncol; c++) {
    // one colour pass reads phi everywhere, fs and phi on its colour, writes phi on its colour
    prof_begin(h, l == 0 ? PC_SWEEP0 : PC_SWEEP_C, w.n * w.S * (1.0 + 2.0 / ncol),
               w.n / ncol * (per_update + (omega != 1.0 || wtab ? 2.0 : 0.0)), w.fp64, s);
    e = (h->nlaunch += 1, launch_sweep_colour(L.d, h->order, L.h, L.dt, L.phi, L.fs, c, omega, st, s, wtab, wlen));
    prof_end(h, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// FP32/BF16 levels (the inner levels of the mixed modes) whose every axis has at
// least tile_min_n intervals, other than the coarsest, use the TMA tile kernels:
// the fused two-colour sweep (7-point) and the fused residual + restriction.
// FP64 levels keep the per-colour passes and the two-kernel restriction: their
// kernels are bound by the FP64 pipe, and the tile kernels' halo recomputation
// adds more FP64 instructions than the HBM traffic they save is worth (measured
// on the 256^3 level: fused restriction 0.42 ms against 0.39 ms).
// tile_min_n < 0 disables the tile kernels.
static const int kTileMinDefault = 16;
bool use_tiles(const ps_ctx* h, const Level& L, int l) {
  const int tmin = h->act.o.tile_min_n == 0 ? kTileMinDefault : h->act.o.tile_min_n;
  if (tmin < 0 || l == h->nlev - 1 || L.dt == DT_F64) return false;
  return L.d.nx >= tmin && L.d.ny >= tmin && L.d.nz >= tmin;
}

// count GS sweeps (omega = 1) on level l, starting and ending in L.phi: pairs of
// out-of-place fused sweeps phi -> phib -> phi on tiled 7-point levels, colour
// passes otherwise (and for an odd last sweep).  skip_first: the first colour
// pass of the first sweep has already run (colour-pass levels only).
cudaError_t smooth(ps_ctx* h, Level& L, int l, int count, cudaStream_t s, bool skip_first = false) {
  cudaError_t e = cudaSuccess;
  int done = 0;
  if (skip_first && count >= 1) {
    if ((e = sweep_level(h, L, l, 1.0, nullptr, s, nullptr, 0, 1)) != cudaSuccess) return e;
    done = 1;
  }
  if (!skip_first && L.phib && h->order == 2 && use_tiles(h, L, l)) {
    const Work w = work_of(L, h->order);
    for (; done + 2 <= count; done += 2) {
      for (int half = 0; half < 2; half++) {
        const void* src = half == 0 ? L.phi : L.phib;
        void* dst = half == 0 ? L.phib : L.phi;
        const int tile = h->act.sweep_tile != 0 ? h->act.sweep_tile : rb_sweep_default_tile(L.dt);
        prof_begin(h, l == 0 ? PC_RBSWEEP0 : PC_RBSWEEP_C, w.n * 3.0 * w.S, w.n * 6.0 * w.G, w.fp64, s, tile);
        e = (h->nlaunch += 1, launch_rb_sweep(L.d, h->order, L.h, L.dt, src, dst, L.fs, nullptr, &h->st->fault, s, tile));
        prof_end(h, s);
        if (e != cudaSuccess) return e;
      }
    }
  }
  for (; done < count; done++)
    if ((e = sweep_level(h, L, l, 1.0, nullptr, s)) != cudaSuccess) return e;
  return cudaSuccess;
}

// skip_first: the first colour pass of level l's pre-smoothing has already run
// (the lagged-norm V-cycles run it at the end of the previous iteration).
cudaError_t vcycle(ps_ctx* h, Hier& H, int l, int nu1, int nu2, cudaStream_t s, bool skip_first = false) {
  Level& L = H.lv[l];
  cudaError_t e;
  if (l == h->nlev - 1) {
    const int nunk = L.d.ni() * L.d.nj() * L.d.nk();
    prof_begin(h, PC_COARSE, 0.0, 0.0, 1, s);
    e = (h->nlaunch += 1, launch_coarse_cg(L.d, h->order, L.h, L.dt, L.fs, L.dt, L.phi, COARSE_TOL, nunk, h->st, s));
    prof_end(h, s);
    return e;
  }
  const Work w = work_of(L, h->order);
  if ((e = smooth(h, L, l, nu1, s, skip_first)) != cudaSuccess) return e;
  Level& Cl = H.lv[l + 1];
  if (use_tiles(h, L, l)) {
    const int rtile = h->order == 2 ? (h->act.restrict_tile != 0 ? h->act.restrict_tile : rr_default_tile(L.dt)) : 0;
    if (l == 0) prof_begin(h, PC_RESTRICT_FUSED0, w.n * 2.0 * w.S + w.n / 8.0 * dt_size(Cl.dt), w.n * (6.0 * w.G + 3.0), w.fp64, s, rtile);
    e = (h->nlaunch += 1, launch_resid_restrict(L.d, Cl.d, h->order, L.h, L.dt, L.phi, L.fs, Cl.dt, Cl.fs, 4.0, &h->st->fault, s, rtile));
    if (l == 0) prof_end(h, s);
    if (e != cudaSuccess) return e;
  } else if (nu1 >= 1 && L.dt != DT_BF16) {
    // the pre-smoothing sweeps end with a complete omega = 1 sweep: the last
    // colour's residual is exactly zero and is not evaluated (not for BF16
    // storage, where it is the rounding error of the stored value)
    const double frac = h->order == 2 ? 0.5 : 2.0 / 3.0;
    const bool diag = L.dt == DT_F64 && L.h[0] == L.h[1] && L.h[1] == L.h[2];
    if (l == 0) prof_begin(h, PC_DELTA0, w.n * (w.S * (1.0 + frac) + w.St), w.n * frac * ((diag ? 5.0 * w.G : 6.0 * w.G) + 1.0), w.fp64, s);
    e = (h->nlaunch += 1, launch_delta_after_sweep(L.d, h->order, L.h, L.dt, L.phi, L.fs, L.dt_tmp, L.tmp, s));
    if (l == 0) prof_end(h, s);
    if (e != cudaSuccess) return e;
    // 7-point: the residual is zero on the black nodes, which the restriction skips
    const bool red = h->order == 2;
    if (l == 0)
      prof_begin(h, PC_RESTRICT0, w.n * w.St + w.n / 8.0 * dt_size(Cl.dt), w.n * (red ? kRestrictRedOps : kRestrictOps),
                 w.St == 8.0, s);
    e = (h->nlaunch += 1, red ? launch_restrict_red(L.d, Cl.d, L.dt_tmp, L.tmp, Cl.dt, Cl.fs, 4.0, s)
                              : launch_restrict(L.d, Cl.d, L.dt_tmp, L.tmp, Cl.dt, Cl.fs, 4.0, s));
    if (l == 0) prof_end(h, s);
    if (e != cudaSuccess) return e;
  } else {
    if (l == 0) prof_begin(h, PC_DELTA0, w.n * (2.0 * w.S + w.St), w.n * (6.0 * w.G + 1.0), w.fp64, s);
    e = (h->nlaunch += 1, launch_delta(L.d, h->order, L.h, L.dt, L.phi, L.fs, L.dt_tmp, L.tmp, 1.0, false, nullptr, nullptr, s));
    if (l == 0) prof_end(h, s);
    if (e != cudaSuccess) return e;
    if (l == 0) prof_begin(h, PC_RESTRICT0, w.n * w.St + w.n / 8.0 * dt_size(Cl.dt), w.n * kRestrictOps, w.St == 8.0, s);
    e = (h->nlaunch += 1, launch_restrict(L.d, Cl.d, L.dt_tmp, L.tmp, Cl.dt, Cl.fs, 4.0, s));
    if (l == 0) prof_end(h, s);
    if (e != cudaSuccess) return e;
  }
  if ((e = cudaMemsetAsync(Cl.phi, 0, (size_t)Cl.d.size() * dt_size(Cl.dt), s)) != cudaSuccess) return e;
  if ((e = vcycle(h, H, l + 1, nu1, nu2, s)) != cudaSuccess) return e;
  if (l == 0) prof_begin(h, PC_PROLONG0, w.n * 2.0 * w.S + w.n / 8.0 * dt_size(Cl.dt), w.n * kProlongOps, w.fp64, s);
  e = (h->nlaunch += 1, launch_prolong(L.d, Cl.d, Cl.dt, Cl.phi, L.dt, L.phi, s));
  if (l == 0) prof_end(h, s);
  if (e != cudaSuccess) return e;
  return smooth(h, L, l, nu2, s);
}

// Convergence pass on the finest FP64 level (optionally storing the IR inner RHS).
// after_sweep: the last operation on phi was a complete omega = 1 colour sweep of
// the finest level, so the last colour's residual is exactly zero and only the
// other colours are evaluated.
// initial: the solve's first residual pass straight after cart_prepare; on
// equal spacings, when the set-up copy found the guess's interior zero, the
// norm-only pass is skipped on the device (the residual is then the reference
// vector) and the 7-point refinement pass reads its deltas off fs and the
// ghost values.
cudaError_t norm_pass(ps_ctx* h, double* phi, int mode, int dout, void* out, cudaStream_t s,
                      unsigned long long cond = 0, int chunk = 0, bool after_sweep = false,
                      bool initial = false) {
  const double n = (double)h->d0.ni() * h->d0.nj() * h->d0.nk();
  const int G = h->order / 2;
  const double dd = make_coef<double>(h->d0, h->h0, h->order).d;
  if (after_sweep && out == nullptr) {
    const double frac = h->order == 2 ? 0.5 : 2.0 / 3.0;   // colours evaluated
    const bool diag = h->h0[0] == h->h0[1] && h->h0[1] == h->h0[2];   // diagonal walks
    prof_begin(h, PC_NORM0, n * 8.0 * (1.0 + frac), n * frac * ((diag ? 5.0 * G : 6.0 * G) + 2.0), 1, s);
    int nb = 0;
    cudaError_t e = (h->nlaunch += 1, launch_delta_colours(h->d0, h->order, h->h0, phi, h->fs64, h->partials, &nb, s));
    prof_end(h, s);
    if (e != cudaSuccess) return e;
    return (h->nlaunch += 1, launch_finish_norm(h->partials, nb, dd, mode, h->st, s, cond, chunk));
  }
  if (h->h0[0] == h->h0[1] && h->h0[1] == h->h0[2]) {
    // (j, k) diagonal walks: 5 + 1 FP64 instructions per node (13-point: 10 + 1),
    // + 1 for the FP64 sum of squares
    const double per = h->order == 2 ? 6.0 : 11.0;
    const bool gate = initial && mode == 1 && out == nullptr;
    // 7-point initial pass with a store: from a zero guess its deltas come from
    // fs and the ghost values alone
    const bool zg = initial && mode == 1 && h->order == 2;
    // (the initial passes are not timed: from a zero guess they do little or no work)
    if (!initial) prof_begin(h, PC_NORM0, n * (16.0 + (out ? (double)dt_size(dout) : 0.0)), n * (out ? per : per + 1.0), 1, s);
    int nb = 0;
    DevState* st = out != nullptr || gate ? h->st : nullptr;
    cudaError_t e = (h->nlaunch += 1,
                     h->order == 2 ? launch_delta_diag(h->d0, h->h0, phi, h->fs64, dout, out, st, zg, h->partials, &nb, s)
                                   : launch_delta_diag13(h->d0, h->h0, out ? 3 : 2, phi, h->fs64, dout, out, st,
                                                         h->partials, &nb, s));
    if (!initial) prof_end(h, s);
    if (e != cudaSuccess) return e;
    return (h->nlaunch += 1, launch_finish_norm(h->partials, nb, dd, gate ? 4 : mode, h->st, s, cond, chunk));
  }
  prof_begin(h, PC_NORM0, n * (16.0 + (out ? (double)dt_size(dout) : 0.0)), n * (6.0 * G + 3.0), 1, s);
  cudaError_t e = out ? launch_delta_st(h->d0, h->order, h->h0, DT_F64, phi, h->fs64, dout, out, h->st, h->partials, s)
                      : launch_delta(h->d0, h->order, h->h0, DT_F64, phi, h->fs64, DT_F64, nullptr, 1.0, false, h->partials, nullptr, s);
  prof_end(h, s);
  if (e != cudaSuccess) return e;
  return (h->nlaunch += 1, launch_finish_norm(h->partials, cart_partials_count(h->d0), dd, mode, h->st, s, cond, chunk));
}

ps_status read_state(ps_ctx* h, cudaStream_t s) {
  TRY(cudaMemcpyAsync(h->hst, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  return PS_OK;
}

// Drop the handle's instantiated graphs (they hold the addresses of its
// buffers); they are captured again on next use.
void drop_graphs(ps_ctx* h) {
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& kv : h->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  h->graphs.clear();
  for (auto& kv : h->pgraphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (auto& rec : kv.second.slots) {
      cudaEventDestroy(rec.a);
      cudaEventDestroy(rec.b);
    }
  }
  h->pgraphs.clear();
}

// Grow the norm-partials buffer.  A reallocation invalidates every graph that
// captured the old address, so those are dropped with it.
ps_status ensure_partials(ps_ctx* h, int nblk) {
  if (nblk <= h->npart) return PS_OK;
  drop_graphs(h);
  cudaFree(h->partials);
  h->partials = nullptr;
  TRY(cudaMalloc(&h->partials, (size_t)nblk * 2 * sizeof(double)));
  h->npart = nblk;
  return PS_OK;
}

// ------------------------------------------------------------------ Cartesian solves
// Multipole boundary (t_mp), scaled right-hand side, state reset and reference
// norm, all enqueued on s without a host round trip.
ps_status cart_prepare(ps_ctx* h, const double* rho, double* phi, double tol, int max_iter,
                       bool own_rhs, cudaStream_t s) {
  TRY(cudaEventRecord(h->ev[0], s));
  if (h->bc.outer == PS_BC_MULTIPOLE) {
    const double n = (double)h->d0.ni() * h->d0.nj() * h->d0.nk();
    const double nf = (double)h->du.size() - n;
    const double W = h->lmax + 1.0;
    prof_begin(h, PC_MOMENTS, n * 8.0, n * W, 1, s);
    cudaError_t e = (h->nlaunch += 4, launch_cart_moments(h->du, h->grid.lo, h->h0, h->bc.origin, rho, &h->mp, s));
    prof_end(h, s);
    TRY(e);
    // one FMA per coefficient of the boundary polynomial (Horner) + about 15 for
    // 1/r, the scaled coordinates and the final product
    prof_begin(h, PC_FACES, nf * 8.0, nf * (W * (W + 1.0) * (W + 2.0) / 6.0 + 15.0), 1, s);
    e = (h->nlaunch += 1, launch_cart_faces(h->du, h->grid.lo, h->h0, h->bc.origin, h->bc.G, h->mp.q, &h->mp, phi, s));
    prof_end(h, s);
    TRY(e);
  }
  TRY(cudaEventRecord(h->ev[1], s));
  Coef<double> cf = make_coef<double>(h->d0, h->h0, h->order);
  const double fscale = -4.0 * M_PI * h->bc.G * cf.inv_d;
  // fs and the partials of the reference norm ||f - A phi0||, phi0 = boundary
  // data only (the compact schemes form R_h f and their reference norm themselves)
  if (!own_rhs)
    TRY((h->nlaunch += 1, launch_scale_rhs_ref(h->d0, h->du, h->order, h->h0, fscale, rho, phi, h->fs64,
                                               h->partials, s)));
  TRY((h->nlaunch += 1, launch_init_state(h->st, tol, max_iter, s)));
  // iterate on the handle's own (pitched) copy of phi: captured loop graphs reference it
  TRY((h->nlaunch += 1, launch_copy_guess(h->d0, h->du, phi, h->phi0, h->st, s)));
  if (own_rhs) return PS_OK;
  TRY((h->nlaunch += 1, launch_finish_norm(h->partials, cart_partials_count(h->d0), cf.d, 0, h->st, s)));
  return PS_OK;
}

static const int MG_CHUNK = 32, KRYLOV_GRAPH_CHUNK = 64;

// Each begin_* enqueues the initial residual pass and installs the iteration
// body (one V-cycle / refinement step / SOR step / Krylov iteration) that the
// step calls repeat.
ps_status begin_mg64(ps_ctx* h, const ps_solve_opts* o, cudaStream_t s) {
  ps_status r = build_hier(h, 0, &h->h64);
  if (r != PS_OK) return r;
  Hier* H = &h->h64;
  double* phi = h->phi0;
  H->lv[0].phi = phi;
  TRY(norm_pass(h, phi, 1, DT_F64, nullptr, s, 0, 0, false, true));
  const int nu1 = o->nu1, nu2 = o->nu2;
  // 7-point on equal spacings with nu1, nu2 >= 1: the convergence check of
  // V-cycle n lags into the first colour pass of V-cycle n + 1 (that pass's
  // x_GS - x_old on colour 0 is V-cycle n's whole residual, colour 1's being
  // zero after the post-smoothing), so the iteration body is
  //   [V-cycle n without its first colour pass] [first colour pass of n + 1,
  //   saving the old colour-0 values and forming the norm of n] [check of n].
  // Each step opens with that first pass (the prologue, skipped once done)
  // and closes by putting back the saved values (the epilogue): the state a
  // step leaves is that of the last V-cycle checked, as without the lag.
  Level& L0 = H->lv[0];
  const bool lag = h->order == 2 && h->h0[0] == h->h0[1] && h->h0[1] == h->h0[2] && nu1 >= 1 && nu2 >= 1 &&
                   h->nlev >= 2 && L0.tmp != nullptr && L0.dt_tmp == DT_F64 && h->d0.sy() % 2 == 0 &&
                   h->d0.sz() % 2 == 0;   // the saved values are packed at node index / 2
  if (lag) {
    double* save = (double*)L0.tmp;
    const double dd = make_coef<double>(h->d0, h->h0, 2).d;
    h->act.body = [h, H, phi, save, nu1, nu2, dd](unsigned long long cond, int chunk, cudaStream_t q) -> cudaError_t {
      cudaError_t e = vcycle(h, *H, 0, nu1, nu2, q, true);
      if (e != cudaSuccess) return e;
      const double n = (double)h->d0.ni() * h->d0.nj() * h->d0.nk();
      int nb = 0;
      prof_begin(h, PC_NORM0, n * 8.0 * 2.0, n * 0.5 * 7.0, 1, q);
      e = (h->nlaunch += 1, launch_sweep_lag(h->d0, h->h0, phi, h->fs64, save, true, h->st, h->partials, &nb, q));
      prof_end(h, q);
      if (e != cudaSuccess) return e;
      return (h->nlaunch += 1, launch_finish_norm(h->partials, nb, dd, 2, h->st, q, cond, chunk));
    };
    h->act.prologue = [h, phi, save](cudaStream_t q) -> cudaError_t {
      return (h->nlaunch += 1, launch_sweep_lag(h->d0, h->h0, phi, h->fs64, save, false, h->st, nullptr, nullptr, q));
    };
    h->act.epilogue = [h, phi, save](cudaStream_t q) -> cudaError_t {
      return (h->nlaunch += 1, launch_restore_colour0(h->d0, phi, save, h->st, q));
    };
  } else {
    h->act.body = [h, H, phi, nu1, nu2](unsigned long long cond, int chunk, cudaStream_t q) -> cudaError_t {
      cudaError_t e = vcycle(h, *H, 0, nu1, nu2, q);
      if (e != cudaSuccess) return e;
      return norm_pass(h, phi, 2, DT_F64, nullptr, q, cond, chunk, nu2 >= 1);
    };
  }
  h->act.key = std::string(lag ? "mg64lag:" : "mg64:") + std::to_string(nu1) + ":" + std::to_string(nu2) + ":" +
               std::to_string(o->tile_min_n);
  h->act.chunk = MG_CHUNK;
  // lagged: profiling steps also run up to a chunk of iterations (the state is
  // read after each), so that the prologue and the restore stay once per step
  h->act.plain_chunk = lag ? MG_CHUNK : 1;
  return PS_OK;
}

ps_status begin_ir(ps_ctx* h, const ps_solve_opts* o, cudaStream_t s) {
  const int p = o->prec == PS_MIXED_BF16 ? 1 : 0;
  ps_status r = build_hier(h, p + 1, &h->hmx[p]);
  if (r != PS_OK) return r;
  Hier* H = &h->hmx[p];
  Level* L0 = &H->lv[0];
  double* phi = h->phi0;
  const int inner = std::max(1, o->inner_cycles);
  TRY(norm_pass(h, phi, 1, L0->dt, L0->fs, s, 0, 0, false, true));
  const int nu1 = o->nu1, nu2 = o->nu2;
  h->act.body = [h, H, L0, phi, nu1, nu2, inner](unsigned long long cond, int chunk, cudaStream_t q) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(L0->phi, 0, (size_t)L0->d.size() * dt_size(L0->dt), q);
    for (int c = 0; c < inner && e == cudaSuccess; c++) e = vcycle(h, *H, 0, nu1, nu2, q);
    if (e != cudaSuccess) return e;
    const double n = (double)h->d0.ni() * h->d0.nj() * h->d0.nk();
    prof_begin(h, PC_CORRECT0, n * (16.0 + dt_size(L0->dt)), n * 2.0, 1, q);
    e = (h->nlaunch += 1, launch_correct(h->d0, L0->dt, L0->phi, 1.0, phi, h->st, q));
    prof_end(h, q);
    if (e != cudaSuccess) return e;
    return norm_pass(h, phi, 2, L0->dt, L0->fs, q, cond, chunk);
  };
  h->act.key = "ir" + std::to_string(p) + ":" + std::to_string(nu1) + ":" + std::to_string(nu2) +
               ":" + std::to_string(inner) + ":" + std::to_string(o->tile_min_n) + ":" +
               std::to_string(h->act.sweep_tile) + ":" + std::to_string(h->act.restrict_tile);
  h->act.chunk = MG_CHUNK;
  h->act.plain_chunk = 1;
  h->act.inner_per_iter = inner;
  return PS_OK;
}

// Eq. 4: Jacobi spectral radius of the Cartesian grid (interval counts and spacings).
double rjac_cartesian(const ps_ctx* h) {
  const int n[3] = {h->d0.nx, h->d0.ny, h->d0.nz};
  double num = 0.0, den = 0.0;
  for (int a = 0; a < 3; a++) {
    const double w = 1.0 / (h->h0[a] * h->h0[a]);
    num += std::cos(M_PI / n[a]) * w;
    den += w;
  }
  return num / den;
}

// Weights of Eq. omega_n from n = 1 until the sequence stops changing in FP64
// (or 65536 entries), one per colour pass; the kernels keep the last entry.
ps_status sor_chebyshev_table(ps_ctx* h, double rj) {
  if (h->sor_wtab) return PS_OK;   // fixed by the grid
  std::vector<double> w;
  double v = 1.0 / (1.0 - rj * rj / 2.0);
  for (int n = 0; n < 65536; n++) {
    w.push_back(v);
    const double nv = 1.0 / (1.0 - rj * rj * v / 4.0);
    if (nv == v) break;
    v = nv;
  }
  ps_status r = alloc_zero((void**)&h->sor_wtab, w.size() * sizeof(double), &h->bytes);
  if (r != PS_OK) return r;
  TRY(cudaMemcpy(h->sor_wtab, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  h->sor_wlen = (int)w.size();
  return PS_OK;
}

ps_status begin_sor(ps_ctx* h, const ps_solve_opts* o, cudaStream_t s) {
  double* phi = h->phi0;
  TRY(norm_pass(h, phi, 1, DT_F64, nullptr, s, 0, 0, false, true));
  Level L0;
  L0.d = h->d0;
  for (int a = 0; a < 3; a++) L0.h[a] = h->h0[a];
  L0.phi = phi;
  L0.fs = h->fs64;
  const double rj = rjac_cartesian(h);
  double omega = o->omega;
  if (o->sor_schedule == PS_SOR_OPTIMAL) omega = 2.0 / (1.0 + std::sqrt(1.0 - rj * rj));
  const double* wtab = nullptr;
  int wlen = 0;
  if (o->sor_schedule == PS_SOR_CHEBYSHEV) {
    ps_status r = sor_chebyshev_table(h, rj);
    if (r != PS_OK) return r;
    wtab = h->sor_wtab;
    wlen = h->sor_wlen;
  }
  h->act.body = [h, L0, phi, omega, wtab, wlen](unsigned long long cond, int chunk, cudaStream_t q) mutable -> cudaError_t {
    cudaError_t e = sweep_level(h, L0, 0, omega, h->st, q, wtab, wlen);
    if (e != cudaSuccess) return e;
    return norm_pass(h, phi, 2, DT_F64, nullptr, q, cond, chunk);
  };
  char key[64];
  if (wtab) snprintf(key, sizeof(key), "sor:chebyshev");
  else snprintf(key, sizeof(key), "sor:%.17g", omega);
  h->act.key = key;
  h->act.chunk = KRYLOV_GRAPH_CHUNK;
  h->act.plain_chunk = KRYLOV_CHUNK;
  return PS_OK;
}

ps_status begin_cg(ps_ctx* h, cudaStream_t s) {
  ps_status r;
  const size_t n = (size_t)h->d0.size();
  if (!h->cg_r) {
    if ((r = alloc_zero((void**)&h->cg_r, n * 8, &h->bytes)) != PS_OK) return r;
    if ((r = alloc_zero((void**)&h->cg_p, n * 8, &h->bytes)) != PS_OK) return r;
    if ((r = alloc_zero((void**)&h->cg_q, n * 8, &h->bytes)) != PS_OK) return r;
  }
  double* phi = h->phi0;
  const int nb = cart_partials_count(h->d0);
  TRY((h->nlaunch += 1, launch_cg_init(h->d0, h->order, h->h0, phi, h->fs64, h->cg_r, h->cg_p, h->partials, nullptr, s)));
  TRY((h->nlaunch += 1, launch_cg_scalar(h->partials, nb, 2, h->st, s)));
  h->act.body = [h, phi, nb](unsigned long long cond, int chunk, cudaStream_t q) -> cudaError_t {
    const double nn = (double)h->d0.ni() * h->d0.nj() * h->d0.nk();
    cudaError_t e;
    prof_begin(h, PC_KRYLOV, nn * 16.0, nn * (6.0 * (h->order / 2) + 3.0), 1, q);
    e = (h->nlaunch += 1, launch_cg_apply(h->d0, h->order, h->h0, h->cg_p, h->cg_q, h->partials, h->st, q));
    prof_end(h, q);
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_cg_scalar(h->partials, nb, 0, h->st, q));
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_cg_update(h->d0, phi, h->cg_r, h->cg_p, h->cg_q, h->partials, h->st, q));
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_cg_scalar(h->partials, nb, 1, h->st, q, cond, chunk));
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_cg_pupdate(h->d0, h->cg_r, h->cg_p, h->st, q));
    return e;
  };
  h->act.key = "cg";
  h->act.chunk = KRYLOV_GRAPH_CHUNK;
  h->act.plain_chunk = KRYLOV_CHUNK;
  return PS_OK;
}

// ------------------------------------------------------------------ compact stencils + SPAI MG
// Table 1: omega, alpha, beta, gamma, delta of the SPAI smoother M of Eq.
// Smoother for compact orders 2, 4, 6.  The order-6 row prints delta equal to
// its mu (a garbled cell); delta = 0.0151 is the value that minimises the local
// Fourier smoothing factor with the printed omega, alpha, beta and gamma.
static const double kSpai[3][5] = {{1.3699, 0.1432, 0.0284, 0.0081, 0.0025},
                                   {0.9363, 0.2807, 0.0329, 0.0166, 0.0044},
                                   {0.3543, 0.7064, 0.1005, 0.0363, 0.0151}};
static const double kCompactCoarseTol = 1e-2;   // coarsest CG, as the geometric MG

struct CompactLevels {
  std::vector<W27> A, M;
  std::vector<double> omega;
};

// Level operators of the compact multigrid for the spacings hl of its levels
// (finest first): compact L_h on the finest, Galerkin products below, the
// SPAI smoother of Table 1 scaled by h_l^2 on every level.
static CompactLevels make_compact_levels(int order, const std::vector<double>& hl) {
  CompactLevels C;
  const double* k = kSpai[order / 2 - 1];
  for (size_t l = 0; l < hl.size(); l++) {
    C.A.push_back(l == 0 ? compact_lhs(order, hl[0]) : galerkin27(C.A.back()));
    C.M.push_back(W27{{k[1] * hl[l] * hl[l], k[2] * hl[l] * hl[l], k[3] * hl[l] * hl[l], k[4] * hl[l] * hl[l]}});
    C.omega.push_back(k[0]);
  }
  return C;
}

// One V-cycle of the compact multigrid (Sec. 2.1.3): SPAI steps
// u -= omega M (b - A u), residual, full weighting into the coarse right-hand
// side, the coarse error from zero, trilinear correction, SPAI steps; the
// coarsest level by CG.  Level l: u = phi, b = fs, r = tmp.
cudaError_t vcycle_compact(ps_ctx* h, Hier* H, const CompactLevels& C, int l, int nu1, int nu2, cudaStream_t s) {
  Level& L = H->lv[l];
  const int last = (int)H->lv.size() - 1;
  const int dt = L.dt;   // DT_F64 (FP64 multigrid) or DT_F32 (inner cycles of the refinement)
  const double S = (double)dt_size(dt);
  const int fp64 = dt == DT_F64;
  void* u = L.phi;
  void* b = L.fs;
  const DevState* st = h->st;
  cudaError_t e;
  if (l == last) {
    prof_begin(h, PC_COARSE, 0.0, 0.0, 1, s);
    e = (h->nlaunch += 1, launch_c27_coarse_cg_dt(L.d, C.A[l], dt, b, u, kCompactCoarseTol, st, s));
    prof_end(h, s);
    return e;
  }
  void* r = L.tmp;
  // FP32 levels smooth out of place, alternating between phi and phib; u is
  // the array that holds the current iterate
  void* ub = fp64 ? nullptr : L.phib;
  const double n = (double)L.d.ni() * L.d.nj() * L.d.nk();
  // residual pass: FP64 levels march z through L1 (four rows per thread), FP32
  // levels run the register-blocked TMA march of the smoothing step
  auto resid = [&](void* out) -> cudaError_t {
    if (fp64) return launch_c27_resid_dt(L.d, C.A[l], (const double*)u, (const double*)b, DT_F64, out, nullptr, st, s);
    return launch_c27_resid_f32(L.d, C.A[l], (const float*)u, (const float*)b, (float*)out, st, &h->st->fault, s);
  };
  auto smooth = [&](int steps) -> cudaError_t {
    for (int it = 0; it < steps; it++) {
      cudaError_t e2;
      if (!fp64) {
        // residual and SPAI step in one pass: reads u and b, writes the other array
        prof_begin(h, l == 0 ? PC_SWEEP0 : PC_SWEEP_C, n * 3.0 * S, n * 32.0, 0, s);
        e2 = (h->nlaunch += 1, launch_c27_smooth(L.d, C.A[l], C.M[l], C.omega[l], (const float*)u,
                                                 (const float*)b, (float*)ub, st, &h->st->fault, s));
        prof_end(h, s);
        if (e2 != cudaSuccess) return e2;
        std::swap(u, ub);
        continue;
      }
      prof_begin(h, l == 0 ? PC_DELTA0 : PC_SWEEP_C, n * 3.0 * S, n * 16.0, fp64, s);
      e2 = (h->nlaunch += 1, resid(r));
      prof_end(h, s);
      if (e2 != cudaSuccess) return e2;
      prof_begin(h, l == 0 ? PC_SWEEP0 : PC_SWEEP_C, n * 3.0 * S, n * 16.0, fp64, s);
      e2 = (h->nlaunch += 1, launch_c27_spai(L.d, C.M[l], C.omega[l], (const double*)r, (double*)u, st, s));
      prof_end(h, s);
      if (e2 != cudaSuccess) return e2;
    }
    return cudaSuccess;
  };
  if ((e = smooth(nu1)) != cudaSuccess) return e;
  if (l == 0) prof_begin(h, PC_DELTA0, n * 3.0 * S, n * 16.0, fp64, s);
  e = (h->nlaunch += 1, resid(r));
  if (l == 0) prof_end(h, s);
  if (e != cudaSuccess) return e;
  Level& Cl = H->lv[l + 1];
  if (l == 0) prof_begin(h, PC_RESTRICT0, n * S * 9.0 / 8.0, n * kRestrictOps, fp64, s);
  e = (h->nlaunch += 1, launch_restrict(L.d, Cl.d, dt, r, Cl.dt, Cl.fs, 1.0, s));
  if (l == 0) prof_end(h, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(Cl.phi, 0, (size_t)Cl.d.size() * dt_size(Cl.dt), s)) != cudaSuccess) return e;
  if ((e = vcycle_compact(h, H, C, l + 1, nu1, nu2, s)) != cudaSuccess) return e;
  if (l == 0) prof_begin(h, PC_PROLONG0, n * S * 17.0 / 8.0, n * kProlongOps, fp64, s);
  e = (h->nlaunch += 1, launch_prolong(L.d, Cl.d, Cl.dt, Cl.phi, dt, u, s));
  if (l == 0) prof_end(h, s);
  if (e != cudaSuccess) return e;
  if ((e = smooth(nu2)) != cudaSuccess) return e;
  // an odd number of out-of-place steps leaves the iterate in phib
  if (u != L.phi) e = cudaMemcpyAsync(L.phi, u, (size_t)L.d.size() * dt_size(dt), cudaMemcpyDeviceToDevice, s);
  return e;
}

// b = R_h (4 pi G rho), then the initial residual r (stored as dt_r) and the
// reference norm ||b - A u0|| in one pass; the state takes the reference
// first, then the initial relative residual.
static cudaError_t compact_prologue(ps_ctx* h, int order, const W27& A0, const double* rho, const double* phi,
                                    double* b, int dt_r, void* r, int nb, cudaStream_t s) {
  const double n = (double)h->d0.ni() * h->d0.nj() * h->d0.nk();
  prof_begin(h, PC_RHS0, n * 16.0, n * (order == 6 ? 19.0 : 12.0), 1, s);
  cudaError_t e = (h->nlaunch += 1, launch_c27_rhs(h->d0, h->du, order, rho, 4.0 * M_PI * h->bc.G, b, s));
  prof_end(h, s);
  if (e != cudaSuccess) return e;
  prof_begin(h, PC_NORM0, n * (16.0 + (double)dt_size(dt_r)), n * 18.0, 1, s);
  e = (h->nlaunch += 1, launch_c27_init(h->d0, A0, phi, b, dt_r, r, h->partials, s));
  prof_end(h, s);
  if (e != cudaSuccess) return e;
  if ((e = (h->nlaunch += 1, launch_finish_norm(h->partials + 2 * nb, nb, 1.0, 0, h->st, s))) != cudaSuccess) return e;
  return (h->nlaunch += 1, launch_finish_norm(h->partials, nb, 1.0, 1, h->st, s));
}

ps_status begin_mg_compact(ps_ctx* h, const double* rho, const ps_solve_opts* o, cudaStream_t s) {
  ps_status r = build_hier(h, 0, &h->h64);
  if (r != PS_OK) return r;
  Hier* H = &h->h64;
  double* phi = h->phi0;
  H->lv[0].phi = phi;
  const int order = o->compact_order;
  std::vector<double> hl;
  for (int l = 0; l < h->nlev; l++) hl.push_back(H->lv[l].h[0]);
  auto C = std::make_shared<CompactLevels>(make_compact_levels(order, hl));
  const int nb = c27_blocks(h->d0);
  if ((r = ensure_partials(h, 2 * nb)) != PS_OK) return r;
  double* b = h->fs64;
  double* rr = (double*)H->lv[0].tmp;
  // b = R_h (4 pi G rho); initial residual and reference ||b - A u0|| (u0:
  // boundary data only) in one pass
  TRY(compact_prologue(h, order, C->A[0], rho, phi, b, DT_F64, rr, nb, s));
  const int nu1 = o->nu1, nu2 = o->nu2;
  h->act.body = [h, H, C, phi, b, rr, nb, nu1, nu2](unsigned long long cond, int chunk, cudaStream_t q) -> cudaError_t {
    cudaError_t e = vcycle_compact(h, H, *C, 0, nu1, nu2, q);
    const double n = (double)h->d0.ni() * h->d0.nj() * h->d0.nk();
    if (e == cudaSuccess) {
      prof_begin(h, PC_NORM0, n * 24.0, n * 17.0, 1, q);
      e = (h->nlaunch += 1, launch_c27_resid(h->d0, C->A[0], phi, b, rr, h->partials, h->st, q));
      prof_end(h, q);
    }
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_finish_norm(h->partials, nb, 1.0, 2, h->st, q, cond, chunk));
    return e;
  };
  h->act.key = "mgc:" + std::to_string(order) + ":" + std::to_string(nu1) + ":" + std::to_string(nu2);
  h->act.chunk = MG_CHUNK;
  h->act.plain_chunk = 1;
  return PS_OK;
}

// Compact multigrid inside FP64 iterative refinement: the outer residual
// r = R_h f - L_h phi in FP64 (stored as the FP32 right-hand side of the inner
// cycles), inner V-cycles on L e = r in FP32 storage and arithmetic (the
// 27-point passes are then bound by HBM instead of the FP64 pipe; coarsest CG in
// FP64 arithmetic), phi += e in FP64.  The stopping test is on the FP64 outer
// residual, as for the FP64 multigrid.
ps_status begin_ir_compact(ps_ctx* h, const double* rho, const ps_solve_opts* o, cudaStream_t s) {
  Hier* H = &h->hmx[0];
  ps_status r = build_hier(h, 1, H);
  if (r != PS_OK) return r;
  const int order = o->compact_order;
  std::vector<double> hl;
  for (int l = 0; l < h->nlev; l++) hl.push_back(H->lv[l].h[0]);
  auto C = std::make_shared<CompactLevels>(make_compact_levels(order, hl));
  const int nb = c27_blocks(h->d0);
  if ((r = ensure_partials(h, 2 * nb)) != PS_OK) return r;
  double* phi = h->phi0;
  double* b64 = h->fs64;
  Level& L0 = H->lv[0];
  // the out-of-place smoothing steps take the zero boundary of the inner
  // error equation from the second array of every smoothed level
  for (int l = 0; l + 1 < h->nlev; l++) {
    Level& L = H->lv[l];
    if (!L.phib) return fail(PS_ERR_CUDA, "compact refinement: level %d has no second array", l);
    TRY(cudaMemsetAsync(L.phib, 0, (size_t)L.d.size() * dt_size(L.dt), s));
  }
  TRY(compact_prologue(h, order, C->A[0], rho, phi, b64, DT_F32, L0.fs, nb, s));
  const int nu1 = o->nu1, nu2 = o->nu2, inner = std::max(1, o->inner_cycles);
  h->act.inner_per_iter = inner;
  h->act.body = [h, H, C, phi, b64, nb, nu1, nu2, inner](unsigned long long cond, int chunk, cudaStream_t q) -> cudaError_t {
    Level& L = H->lv[0];
    cudaError_t e = cudaMemsetAsync(L.phi, 0, (size_t)L.d.size() * sizeof(float), q);
    for (int c = 0; c < inner && e == cudaSuccess; c++) e = vcycle_compact(h, H, *C, 0, nu1, nu2, q);
    const double n = (double)h->d0.ni() * h->d0.nj() * h->d0.nk();
    if (e == cudaSuccess) {
      prof_begin(h, PC_CORRECT0, n * 20.0, n, 1, q);
      // the partials carry no max, so the state keeps scale 1 and e is added unscaled
      e = (h->nlaunch += 1, launch_correct(h->d0, DT_F32, L.phi, 1.0, phi, h->st, q));
      prof_end(h, q);
    }
    if (e == cudaSuccess) {
      prof_begin(h, PC_NORM0, n * 20.0, n * 17.0, 1, q);
      e = (h->nlaunch += 1, launch_c27_resid_dt(h->d0, C->A[0], phi, b64, DT_F32, L.fs, h->partials, h->st, q));
      prof_end(h, q);
    }
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_finish_norm(h->partials, nb, 1.0, 2, h->st, q, cond, chunk));
    return e;
  };
  h->act.key = "irc:" + std::to_string(order) + ":" + std::to_string(nu1) + ":" + std::to_string(nu2) + ":" +
               std::to_string(inner);
  h->act.chunk = MG_CHUNK;
  h->act.plain_chunk = 1;
  return PS_OK;
}

// CG preconditioned by multicolour symmetric Gauss-Seidel (Sec. 2.1.2): the CG
// recurrences with z = B^-1 r in the direction and in rho = r.z; stopping on
// the unpreconditioned residual as CG.
ps_status begin_pcg(ps_ctx* h, cudaStream_t s) {
  ps_status r;
  const size_t n = (size_t)h->d0.size();
  if (!h->cg_r) {
    if ((r = alloc_zero((void**)&h->cg_r, n * 8, &h->bytes)) != PS_OK) return r;
    if ((r = alloc_zero((void**)&h->cg_p, n * 8, &h->bytes)) != PS_OK) return r;
    if ((r = alloc_zero((void**)&h->cg_q, n * 8, &h->bytes)) != PS_OK) return r;
  }
  if (!h->cg_z && (r = alloc_zero((void**)&h->cg_z, n * 8, &h->bytes)) != PS_OK) return r;
  const int nbz = pcg_partials_count(h->d0, h->order);
  if ((r = ensure_partials(h, nbz)) != PS_OK) return r;
  double* phi = h->phi0;
  const int nb = cart_partials_count(h->d0);
  TRY((h->nlaunch += 1, launch_cg_init(h->d0, h->order, h->h0, phi, h->fs64, h->cg_r, h->cg_p, h->partials, nullptr, s)));
  TRY((h->nlaunch += 1, launch_cg_scalar(h->partials, nb, 2, h->st, s)));
  TRY((h->nlaunch += pcg_precond_kernels(h->order), launch_pcg_precond(h->d0, h->order, h->h0, h->cg_r, h->cg_z, h->partials, h->st, s)));
  TRY((h->nlaunch += 1, launch_cg_scalar(h->partials, nbz, 5, h->st, s)));
  TRY(cudaMemcpyAsync(h->cg_p, h->cg_z, n * 8, cudaMemcpyDeviceToDevice, s));
  h->act.body = [h, phi, nb, nbz](unsigned long long cond, int chunk, cudaStream_t q) -> cudaError_t {
    const double nn = (double)h->d0.ni() * h->d0.nj() * h->d0.nk();
    const int ncol = h->order == 2 ? 2 : 3;
    cudaError_t e;
    prof_begin(h, PC_KRYLOV, nn * 16.0, nn * (6.0 * (h->order / 2) + 3.0), 1, q);
    e = (h->nlaunch += 1, launch_cg_apply(h->d0, h->order, h->h0, h->cg_p, h->cg_q, h->partials, h->st, q));
    prof_end(h, q);
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_cg_scalar(h->partials, nb, 0, h->st, q));
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_cg_update(h->d0, phi, h->cg_r, h->cg_p, h->cg_q, h->partials, h->st, q));
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_cg_scalar(h->partials, nb, 3, h->st, q, cond, chunk));
    if (e == cudaSuccess) {
      // 2 ncol - 1 colour passes, each reading z around and r on its colour
      prof_begin(h, PC_SWEEP0, nn * 8.0 * (2 * ncol - 1) * (1.0 + 2.0 / ncol),
                 nn / ncol * (2 * ncol - 1) * (6.0 * (h->order / 2) + 1.0), 1, q);
      e = (h->nlaunch += pcg_precond_kernels(h->order), launch_pcg_precond(h->d0, h->order, h->h0, h->cg_r, h->cg_z, h->partials, h->st, q));
      prof_end(h, q);
    }
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_cg_scalar(h->partials, nbz, 4, h->st, q));
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_cg_pupdate(h->d0, h->cg_z, h->cg_p, h->st, q));
    return e;
  };
  h->act.key = "pcg";
  h->act.chunk = KRYLOV_GRAPH_CHUNK;
  h->act.plain_chunk = KRYLOV_CHUNK;
  return PS_OK;
}

// ------------------------------------------------------------------ spherical solves
ps_status sph_vectors(ps_ctx* h, int dt) {
  if (h->sv_dt == dt) return PS_OK;
  const size_t n = (size_t)h->sd.size();
  if (h->sv_dt >= 0) h->bytes -= 8 * n * dt_size(h->sv_dt);
  for (auto& p : h->sv) { cudaFree(p); p = nullptr; }
  h->sv_dt = -1;
  for (int q = 0; q < 8; q++) {
    ps_status r = alloc_zero(&h->sv[q], n * dt_size(dt), &h->bytes);
    if (r != PS_OK) return r;
  }
  h->sv_dt = dt;
  return PS_OK;
}

// Enqueue a BiCGSTAB start (reference and initial residual) with Krylov
// vectors of storage dt and return its iteration body.  x is the FP64 iterate.
// vectors: 0 r, 1 rhat, 2 p, 3 phat, 4 v, 5 s, 6 shat, 7 t
ps_status bicg_start(ps_ctx* h, int dt, const double* rho, double fscale, double* x, DevState* st,
                     double tol, int max_iter, cudaStream_t s, Body* body, double drop = 0.01,
                     int restart_on_replace = 0) {
  int nb = 0;
  void** v = h->sv;
  TRY((h->nlaunch += 1, launch_init_state(st, tol, max_iter, s)));
  TRY((h->nlaunch += 1, launch_bicg_resid(h->sd, h->stab, dt, 0, rho, fscale, x, nullptr, nullptr, nullptr, nullptr, h->partials, &nb, s)));
  TRY((h->nlaunch += 1, launch_bicg_start(h->partials, nb, 0, st, s)));
  TRY((h->nlaunch += 1, launch_bicg_resid(h->sd, h->stab, dt, 1, rho, fscale, x, v[0], v[1], v[2], v[3], h->partials, &nb, s)));
  TRY((h->nlaunch += 1, launch_bicg_start(h->partials, nb, 1, st, s, drop, restart_on_replace)));
  if (!h->sz) {
    ps_status r = alloc_zero((void**)&h->sz, (size_t)h->sd.size() * sizeof(double), &h->bytes);
    if (r != PS_OK) return r;
  }
  TRY(cudaMemsetAsync(h->sz, 0, (size_t)h->sd.size() * sizeof(double), s));
  double* z = h->sz;
  *body = [h, dt, rho, fscale, x, z, v, st](unsigned long long cond, int chunk, cudaStream_t q) -> cudaError_t {
    const double n = (double)h->sd.nr * h->sd.nt * h->sd.np;
    const double S = dt == DT_F64 ? 8.0 : 4.0;
    // 21 vector streams of the storage type (apply 3, s 4, apply 3, x/r 6,
    // p 5) plus the FP64 increment z read and written; replacements (a few
    // per hundred iterations) are not counted
    const double bytes = n * (S * 21.0 + 16.0);
    prof_begin(h, PC_KRYLOV, bytes, n * 60.0, dt == DT_F64, q);
    h->nlaunch += bicg_iter_kernels(dt);
    cudaError_t e = launch_bicg_iter(h->sd, h->stab, dt, rho, fscale, x, z, v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], h->partials, st, q, cond, chunk);
    prof_end(h, q);
    return e;
  };
  return PS_OK;
}

// Spherical solve: right-Jacobi BiCGSTAB stopping on true residuals.  PS_FP64
// keeps every vector in FP64; the mixed precisions keep the Krylov vectors in
// FP32 and the iterate, the right-hand side, the replaced residuals and every
// dot product in FP64.
// Spherical red-black SOR (Sec. 2.1.1) in FP64, stopping on ||f - L x|| <=
// tol ||b||, b = f - L(boundary part of x) as for BiCGSTAB.  The weights are
// the given omega, or per node from the local rJ of Eq. local_rjac: omega_opt
// of Eq. 3, or the sequence of Eq. omega_n advanced by every colour pass in two
// alternating buffers (pass colour 0 reads buffer 0 and writes buffer 1).
ps_status begin_sph_sor(ps_ctx* h, const double* rho, double fscale, double* x, double tol,
                        const ps_solve_opts* o, cudaStream_t s) {
  const SphDims d = h->sd;
  ps_status r;
  const int nb = sph_sor2_blocks(d);
  if ((r = ensure_partials(h, std::max(2 * nb, sph_resnorm_blocks(d)))) != PS_OK) return r;
  const size_t nq = (size_t)d.nr * d.nt;
  const int sched = o->sor_schedule;
  if (sched != PS_SOR_FIXED && !h->sph_w)
    if ((r = alloc_zero((void**)&h->sph_w, 2 * nq * sizeof(double), &h->bytes)) != PS_OK) return r;
  if (!h->sph_g)
    if ((r = alloc_zero((void**)&h->sph_g, (size_t)d.size() * sizeof(double), &h->bytes)) != PS_OK) return r;
  int nb0 = 0;
  TRY((h->nlaunch += 1, launch_init_state(h->st, tol, o->max_iter, s)));
  TRY((h->nlaunch += 1, launch_bicg_resid(d, h->stab, DT_F64, 0, rho, fscale, x, nullptr, nullptr, nullptr, nullptr, h->partials, &nb0, s)));
  TRY((h->nlaunch += 1, launch_finish_norm(h->partials, nb0, 1.0, 0, h->st, s)));
  TRY((h->nlaunch += 1, launch_sph_resnorm(d, h->stab, x, rho, fscale, h->partials, &nb0, s)));
  TRY((h->nlaunch += 1, launch_finish_norm(h->partials, nb0, 1.0, 1, h->st, s)));
  TRY((h->nlaunch += 1, launch_sph_gs(d, h->stab, rho, fscale, h->sph_g, s)));
  if (sched != PS_SOR_FIXED)
    TRY((h->nlaunch += 1, launch_sph_sor_weights(d, h->stab, sched == PS_SOR_CHEBYSHEV, h->sph_w, s)));
  double* w0 = h->sph_w;
  double* w1 = h->sph_w ? h->sph_w + nq : nullptr;
  const double omega = o->omega;
  const double* g = h->sph_g;
  // one step: red pass, black pass (with the black nodes' residuals after it),
  // red nodes' residuals, norm and convergence check
  h->act.body = [h, d, g, x, sched, omega, w0, w1, nb](unsigned long long cond, int chunk, cudaStream_t q) -> cudaError_t {
    const double n = (double)d.nr * d.nt * d.np;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < 2 && e == cudaSuccess; c++) {
      const double* wc = sched == PS_SOR_FIXED ? nullptr : (sched == PS_SOR_OPTIMAL || c == 0 ? w0 : w1);
      double* wn = sched == PS_SOR_CHEBYSHEV ? (c == 0 ? w1 : w0) : nullptr;
      // a pass reads x everywhere, g and x on its colour, writes x on its colour;
      // 8 FP64 instructions per red update, 13 (+4 for the residual) per black one
      prof_begin(h, PC_SWEEP0, n * 16.0, n / 2 * (c == 0 ? 8.0 : 17.0), 1, q);
      e = (h->nlaunch += 1, launch_sph_sor2(d, h->stab, x, g, c, omega, wc, wn, c == 1 ? h->partials : nullptr, h->st, q));
      prof_end(h, q);
    }
    if (e == cudaSuccess) {
      prof_begin(h, PC_NORM0, n * 12.0, n / 2 * 14.0, 1, q);
      e = (h->nlaunch += 1, launch_sph_rednorm(d, h->stab, x, g, h->partials + 2 * nb, h->st, q));
      prof_end(h, q);
    }
    if (e == cudaSuccess) e = (h->nlaunch += 1, launch_finish_norm(h->partials, 2 * nb, 1.0, 3, h->st, q, cond, chunk));
    return e;
  };
  char key[64];
  snprintf(key, sizeof(key), "sphsor:%d:%.17g", sched, sched == PS_SOR_FIXED ? omega : 0.0);
  h->act.key = key;
  h->act.chunk = KRYLOV_GRAPH_CHUNK;
  h->act.plain_chunk = KRYLOV_CHUNK;
  return PS_OK;
}

ps_status begin_sph(ps_ctx* h, const double* rho, double* phi_user, double tol, const ps_solve_opts* o,
                    cudaStream_t s) {
  ps_status r;
  TRY(cudaEventRecord(h->ev[0], s));
  const bool inner_mp = h->bc.inner == PS_INNER_MULTIPOLE;
  if (h->bc.outer == PS_BC_MULTIPOLE || inner_mp)
    TRY((h->nlaunch += inner_mp ? 3 : 2, launch_sph_moments(h->sd, h->stab, rho, s)));
  if (h->bc.outer == PS_BC_MULTIPOLE) TRY((h->nlaunch += 1, launch_sph_face(h->sd, h->stab, h->bc.G, phi_user, s)));
  if (inner_mp) TRY((h->nlaunch += 1, launch_sph_face_inner(h->sd, h->stab, h->bc.G, phi_user, s)));
  TRY(cudaEventRecord(h->ev[1], s));
  double* phi = h->phi0;
  TRY(cudaMemcpyAsync(phi, phi_user, (size_t)h->sd.size() * sizeof(double), cudaMemcpyDeviceToDevice, s));
  const double fscale = 4.0 * M_PI * h->bc.G;
  if (o->method == PS_SOR) return begin_sph_sor(h, rho, fscale, phi, tol, o, s);
  h->act.chunk = KRYLOV_GRAPH_CHUNK;
  h->act.plain_chunk = KRYLOV_CHUNK;
  const int dt = o->prec == PS_FP64 ? DT_F64 : DT_F32;
  if ((r = sph_vectors(h, dt)) != PS_OK) return r;
  h->act.key = dt == DT_F64 ? "bicg64" : "bicg32";
  h->act.count_replacements = dt != DT_F64;
  if (dt == DT_F64) return bicg_start(h, dt, rho, fscale, phi, h->st, tol, o->max_iter, s, &h->act.body);
  // FP32 Krylov vectors: iterative refinement.  Each inner FP32 BiCGSTAB runs
  // until its recursive residual has dropped 2^-k-fold (k = inner_cycles, 2 by
  // default: at 256 x 128 x 256 to 1e-8, k = 2, 3, 4, 5, 6 took 1.97, 2.28,
  // 3.72, 3.11, 2.98 s and k = 8 did not converge), then x takes the FP64
  // increments, the FP64 true residual replaces r and a new Krylov process
  // starts from it.
  const int k = o->inner_cycles > 0 ? std::min(o->inner_cycles, 30) : 2;
  return bicg_start(h, dt, rho, fscale, phi, h->st, tol, o->max_iter, s, &h->act.body, std::ldexp(1.0, -k), 1);
}

// ------------------------------------------------------------------ stepping
// Capture the active body into a graph: gate kernel -> while(body).  The gate
// opens the loop only when the state has work left within the step budget;
// the body's last scalar kernel re-evaluates the condition every iteration.
ps_status build_loop_graph(ps_ctx* h, LoopGraph* g) {
  cudaGraph_t graph = nullptr;
  TRY(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault);
  cudaGraphNode_t gate = nullptr;
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(h->cap, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t eg = launch_loop_gate(h->st_active, (unsigned long long)cond, h->cap);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(h->cap, &captured);
    if (eg != cudaSuccess) e = eg;
  }
  size_t nn = 1;
  if (e == cudaSuccess) e = cudaGraphGetNodes(graph, &gate, &nn);
  alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)];
  memset(np_raw, 0, sizeof(np_raw));
  cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_raw);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t wnode;
  if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, graph, &gate, nullptr, 1, &np);
  if (e == cudaSuccess) {
    cudaGraph_t bodyg = np.conditional.phGraph_out[0];
    const long long before = h->nlaunch;
    e = cudaStreamBeginCaptureToGraph(h->cap, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t eb = h->act.body((unsigned long long)cond, 1, h->cap);
      cudaGraph_t captured = nullptr;
      e = cudaStreamEndCapture(h->cap, &captured);
      if (eb != cudaSuccess) e = eb;
    }
    g->body_kernels = h->nlaunch - before;
    h->nlaunch = before;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g->exec = nullptr;
    return fail(PS_ERR_CUDA, "building the %s loop graph: %s", h->act.key.c_str(), cudaGetErrorString(e));
  }
  return PS_OK;
}

// Enqueue up to k more iterations of the active solve on the handle's stream.
ps_status step_active(ps_ctx* h, int k) {
  cudaStream_t s = h->stream;
  ps_status r;
  if (k <= 0) return PS_OK;
  if (h->prof) {
    // Event records cannot sit inside conditional graph bodies, so profiling
    // replays one iteration per launch from a plain graph that carries event
    // record nodes around the hot kernels, after a state read so that no
    // iteration runs past convergence; the events are harvested after each
    // launch (no host gaps between the kernels being timed).
    if ((r = read_state(h, s)) != PS_OK) return r;
    if (h->act.prologue) TRY(h->act.prologue(s));
    ProfGraph& pg = h->pgraphs[h->act.key];
    if (!pg.exec) {
      while (h->ev_pool.size() < 512) {
        cudaEvent_t ev;
        TRY(cudaEventCreate(&ev));
        h->ev_pool.push_back(ev);
      }
      const long long before = h->nlaunch;
      TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
      h->cap_slots = &pg.slots;
      cudaError_t eb = h->act.body(0ull, 0, h->cap);
      h->cap_slots = nullptr;
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
      if (eb != cudaSuccess) e = eb;
      pg.body_kernels = h->nlaunch - before;
      h->nlaunch = before;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&pg.exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        pg.exec = nullptr;
        return fail(PS_ERR_CUDA, "building the profiling graph: %s", cudaGetErrorString(e));
      }
    }
    const int n = std::min(k, h->act.plain_chunk);
    for (int q = 0; q < n && h->hst->done == DONE_NO; q++) {
      TRY(cudaGraphLaunch(pg.exec, s));
      TRY(cudaStreamSynchronize(s));
      h->nlaunch += pg.body_kernels;
      for (auto& rec : pg.slots) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, rec.a, rec.b) != cudaSuccess) {
          (void)cudaGetLastError();   // a slot that did not run leaves no sticky error
          continue;
        }
        ProfAcc& a = h->acc[rec.cls];
        a.n++;
        a.ms += ms;
        a.bytes += rec.bytes;
        a.ops += rec.ops;
        a.fp64 = rec.fp64;
        a.variant = rec.variant;
      }
      if (q + 1 < n && (r = read_state(h, s)) != PS_OK) return r;
    }
    if (h->act.epilogue) TRY(h->act.epilogue(s));
    h->act.plain_steps = true;
    return PS_OK;
  }
  LoopGraph& g = h->graphs[h->act.key];
  if (!g.exec && (r = build_loop_graph(h, &g)) != PS_OK) return r;
  h->act.body_kernels = g.body_kernels;
  TRY((h->nlaunch += 2, launch_set_budget(h->st, k, s)));
  if (h->act.prologue) TRY(h->act.prologue(s));
  TRY(cudaGraphLaunch(g.exec, s));
  if (h->act.epilogue) TRY(h->act.epilogue(s));
  return PS_OK;
}

// Read the active solve's state (waits for its stream).
ps_status poll_active(ps_ctx* h, int* done) {
  const int it0 = h->hst->iter;
  ps_status r = read_state(h, h->stream);
  if (r != PS_OK) return r;
  if (!h->act.plain_steps && h->hst->iter > it0)
    h->nlaunch += h->act.body_kernels * (h->hst->iter - it0);
  h->act.plain_steps = false;
  *done = h->hst->done != DONE_NO;
  return PS_OK;
}

void fill_info(ps_ctx* h, ps_info* info, ps_status st, bool final_) {
  if (!info) return;
  memset(info, 0, sizeof(*info));
  const DevState& d = *h->hst;
  info->iterations = d.iter;
  info->rel_residual = d.rel;
  info->rho_conv = (d.iter > 0 && d.rel0 > 0.0) ? std::pow(d.rel / d.rel0, 1.0 / d.iter) : 0.0;
  info->inner_cycles = h->act.count_replacements ? d.inner_cycles : (long long)d.iter * h->act.inner_per_iter;
  info->coarse_iterations = d.coarse_iter_total;
  info->kernel_launches = h->nlaunch;
  info->status = st;
  float a = 0.f, b = 0.f;
  if (cudaEventElapsedTime(&a, h->ev[0], h->ev[1]) == cudaSuccess) info->t_mp_ms = a;
  if (final_ && cudaEventElapsedTime(&b, h->ev[1], h->ev[2]) == cudaSuccess) info->t_iter_ms = b;
  if (h->bc.outer == PS_BC_MULTIPOLE) {
    const int nq = std::min(81, (h->lmax + 1) * (h->lmax + 1));
    const double* q = h->sph ? h->stab.q : h->mp.q;
    if (q) cudaMemcpy(info->moments, q, nq * sizeof(double), cudaMemcpyDeviceToHost);
  }
}

size_t cart_bytes(const ps_grid* g, int order, int lmax, int prec, bool multipole) {
  std::vector<std::array<int, 3>> lv;
  levels_for(g->n, &lv);
  const int gw = order / 2;
  size_t b = 0;
  Dims d0 = level_dims(lv[0], gw, lv.size() == 1);
  b += (size_t)d0.size() * 8;   // fs64
  for (size_t l = 0; l < lv.size(); l++) {
    const bool last = l + 1 == lv.size();
    Dims d = level_dims(lv[l], gw, last);
    if (prec == PS_FP64) {
      b += (size_t)d.size() * 8 * (l == 0 ? (last ? 0 : 1) : (last ? 2 : 3));
    } else {
      // phi, fs, the delta buffer and (7-point) the fused sweeps' second phi
      const size_t s = (l == 0 && prec == PS_MIXED_BF16) ? 2 : 4;
      b += (size_t)d.size() * (2 * s + (last ? 0 : 4 + (order == 2 ? s : 0)));
    }
  }
  if (multipole) b += cart_multipole_bytes(make_dims(g->n[0], g->n[1], g->n[2], gw), lmax);
  b += (size_t)cart_partials_count(d0) * 16 + 2 * sizeof(DevState);
  return b;
}


// ====================================================================== batched executor (host)
struct BSlotHost {
  ps_ctx* h = nullptr;
  double* phi_user = nullptr;
  long long iters_at_add = 0;
};

}  // namespace

struct ps_batch_ctx {
  int cap = 0, order = 2, prec = 0, nu1 = 2, nu2 = 2, inner = 1, nlev_max = 0;
  cudaStream_t stream = nullptr, capstream = nullptr;
  std::vector<BSlotHost> slots;
  std::vector<BSlot> hslots;
  BSlot* dslots = nullptr;
  BItem* ditems = nullptr;
  size_t items_cap = 0;
  BList* dlists = nullptr;
  int* dstatus = nullptr;
  int* hstatus = nullptr;   // pinned
  std::map<int, cudaGraphExec_t> graphs;   // by iterations per step
  size_t graph_smem = 0;                   // coarsest-CG shared memory the graphs were built with
  bool dirty = true;
  int kernels_per_iter = 0;
};

namespace {

void destroy_batch_graphs(ps_batch_ctx* b) {
  for (auto& kv : b->graphs)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

// Rebuild the work lists and upload the slot descriptors (after a change of
// the batch's composition).
ps_status batch_rebuild(ps_batch_ctx* b) {
  const int L = PS_BMAX_LEVELS;
  std::vector<std::vector<BItem>> lists(BL_NKINDS * L);
  std::vector<int> totals(BL_NKINDS * L, 0);
  auto push = [&](int list, int si, int level, int gx, int gy, int gz) {
    const int tiles = gx * gy * gz;
    lists[list].push_back({si, level, totals[list], tiles, gx, gy});
    totals[list] += tiles;
  };
  size_t smem = 8;
  for (int si = 0; si < b->cap; si++) {
    BSlot& sd = b->hslots[si];
    if (!sd.active) continue;
    ps_ctx* h = b->slots[si].h;
    const int nl = sd.nlev;
    int gx, gy, gz;
    for (int l = 0; l + 1 < nl; l++) {
      batch_tiles_sweep(sd.lv[l].d, b->order, sd.lv[l].zc, &gx, &gy, &gz);
      push(BL_SWEEP * L + l, si, l, gx, gy, gz);
      batch_tiles_points(sd.lv[l + 1].d, sd.lv[l + 1].zc, &gx, &gy, &gz);
      push(BL_COARSE_PT * L + l, si, l, gx, gy, gz);
      batch_tiles_cells(sd.lv[l + 1].d, sd.lv[l + 1].zc, &gx, &gy, &gz);
      push(BL_CELLS * L + l, si, l, gx, gy, gz);
    }
    push(BL_CG * L + (nl - 1), si, nl - 1, 1, 1, 1);
    smem = std::max(smem, coarse_cg_smem_bytes(sd.lv[nl - 1].d));
    if (b->prec == 0) {
      batch_tiles_sweep(sd.lv[0].d, b->order, sd.lv[0].zc, &gx, &gy, &gz);
      push(BL_NORM0 * L, si, 0, gx, gy, gz);
    } else {
      batch_tiles_points(sd.lv[0].d, sd.lv[0].zc, &gx, &gy, &gz);
      push(BL_PT0 * L, si, 0, gx, gy, gz);
    }
    sd.nparts = gx * gy * gz;   // one norm partial per level-0 tile
    ps_status r = ensure_partials(h, sd.nparts);
    if (r != PS_OK) return r;
    sd.partials = h->partials;
    push(BL_SLOTS * L, si, 0, 1, 1, 1);
  }
  std::vector<BItem> items;
  std::vector<BList> heads(BL_NKINDS * L);
  for (size_t q = 0; q < lists.size(); q++) {
    heads[q].off = (int)items.size();
    heads[q].count = (int)lists[q].size();
    heads[q].total = totals[q];
    heads[q].pad_ = 0;
    items.insert(items.end(), lists[q].begin(), lists[q].end());
  }
  if (items.size() > b->items_cap) {
    // the graphs hold the item array's address: rebuild them with the new one
    TRY(cudaStreamSynchronize(b->stream));
    destroy_batch_graphs(b);
    cudaFree(b->ditems);
    b->ditems = nullptr;
    b->items_cap = std::max<size_t>(items.size() * 2, 1024);
    TRY(cudaMalloc(&b->ditems, b->items_cap * sizeof(BItem)));
  }
  if (smem > b->graph_smem) {
    TRY(cudaStreamSynchronize(b->stream));
    destroy_batch_graphs(b);
    b->graph_smem = smem;
  }
  if (!items.empty())
    TRY(cudaMemcpyAsync(b->ditems, items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice, b->stream));
  TRY(cudaMemcpyAsync(b->dlists, heads.data(), heads.size() * sizeof(BList), cudaMemcpyHostToDevice, b->stream));
  TRY(cudaMemcpyAsync(b->dslots, b->hslots.data(), b->hslots.size() * sizeof(BSlot), cudaMemcpyHostToDevice, b->stream));
  // the host vectors are pageable: the copies above complete before returning
  b->dirty = false;
  return PS_OK;
}

// One V-cycle of every active solve over the work lists (levels are indexed
// from the finest; a solve's coarsest level is solved where it occurs).
cudaError_t batch_vcycle(ps_batch_ctx* b, int dt, cudaStream_t s) {
  const BArgs a{b->dslots, b->ditems, b->dlists};
  const int L = PS_BMAX_LEVELS, ncol = b->order == 2 ? 2 : 3;
  cudaError_t e;
  for (int l = 0; l + 1 < b->nlev_max; l++) {
    for (int it = 0; it < b->nu1; it++)
      for (int c = 0; c < ncol; c++)
        if ((e = launch_b_sweep(a, b->order, dt, BL_SWEEP * L + l, c, s)) != cudaSuccess) return e;
    if ((e = launch_b_delta_skip(a, b->order, dt, BL_SWEEP * L + l, s)) != cudaSuccess) return e;
    if ((e = launch_b_restrict(a, dt, BL_COARSE_PT * L + l, s)) != cudaSuccess) return e;
    if ((e = launch_b_coarse(a, b->order, dt, BL_CG * L + l + 1, b->cap, b->graph_smem, COARSE_TOL, s)) != cudaSuccess) return e;
  }
  for (int l = b->nlev_max - 2; l >= 0; l--) {
    if ((e = launch_b_prolong(a, dt, BL_CELLS * L + l, s)) != cudaSuccess) return e;
    for (int it = 0; it < b->nu2; it++)
      for (int c = 0; c < ncol; c++)
        if ((e = launch_b_sweep(a, b->order, dt, BL_SWEEP * L + l, c, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One iteration of every active solve: a V-cycle and its convergence check
// (FP64), or a refinement step (mixed FP32).
cudaError_t batch_iteration(ps_batch_ctx* b, cudaStream_t s) {
  const BArgs a{b->dslots, b->ditems, b->dlists};
  const int L = PS_BMAX_LEVELS;
  cudaError_t e;
  if (b->prec == 0) {
    if ((e = batch_vcycle(b, DT_F64, s)) != cudaSuccess) return e;
    if ((e = launch_b_norm(a, b->order, BL_NORM0 * L, s)) != cudaSuccess) return e;
    return launch_b_finish(a, BL_SLOTS * L, b->cap, s);
  }
  if ((e = launch_b_zero(a, DT_F32, BL_PT0 * L, s)) != cudaSuccess) return e;
  for (int c = 0; c < b->inner; c++)
    if ((e = batch_vcycle(b, DT_F32, s)) != cudaSuccess) return e;
  if ((e = launch_b_correct(a, BL_PT0 * L, s)) != cudaSuccess) return e;
  if ((e = launch_b_delta_ir(a, b->order, BL_PT0 * L, s)) != cudaSuccess) return e;
  return launch_b_finish(a, BL_SLOTS * L, b->cap, s);
}

ps_status batch_graph(ps_batch_ctx* b, int iters, cudaGraphExec_t* out) {
  auto it = b->graphs.find(iters);
  if (it != b->graphs.end()) {
    *out = it->second;
    return PS_OK;
  }
  TRY(cudaStreamBeginCapture(b->capstream, cudaStreamCaptureModeThreadLocal));
  cudaError_t eb = cudaSuccess;
  for (int k = 0; k < iters && eb == cudaSuccess; k++) eb = batch_iteration(b, b->capstream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->capstream, &graph);
  if (eb != cudaSuccess) e = eb;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(PS_ERR_CUDA, "building the batch step graph: %s", cudaGetErrorString(e));
  b->graphs[iters] = exec;
  *out = exec;
  return PS_OK;
}

void batch_level_desc(ps_ctx* h, const Level& L, BLevel* out) {
  memset(out, 0, sizeof(*out));
  out->d = L.d;
  out->cf64 = make_coef<double>(L.d, L.h, h->order);
  out->cf32 = make_coef<float>(L.d, L.h, h->order);
  out->phi = L.phi;
  out->fs = L.fs;
  out->tmp = L.tmp;
  out->dt = L.dt;
  out->iso = (L.h[0] == L.h[1] && L.h[1] == L.h[2]) ? 1 : 0;
  out->zc = batch_zchunk(L.d);
}
}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* poisson_last_error(void) { return g_err.c_str(); }

ps_status poisson_compact_operators(int order, double h, int nlevels, double* a, double* m, double* omega) {
  if (order != 2 && order != 4 && order != 6)
    return fail(PS_ERR_INVALID_ARG, "compact order must be 2, 4 or 6 (got %d)", order);
  if (!(h > 0.0) || !std::isfinite(h)) return fail(PS_ERR_INVALID_ARG, "h must be positive and finite");
  if (nlevels < 1 || nlevels > 30) return fail(PS_ERR_INVALID_ARG, "nlevels must be in 1..30 (got %d)", nlevels);
  if (!a) return fail(PS_ERR_INVALID_ARG, "a must not be NULL");
  std::vector<double> hl;
  for (int l = 0; l < nlevels; l++) hl.push_back(std::ldexp(h, l));
  const CompactLevels C = make_compact_levels(order, hl);
  for (int l = 0; l < nlevels; l++) {
    for (int c = 0; c < 4; c++) {
      a[4 * l + c] = C.A[l].w[c];
      if (m) m[4 * l + c] = C.M[l].w[c];
    }
    if (omega) omega[l] = C.omega[l];
  }
  return PS_OK;
}

ps_status poisson_set_tuning(ps_handle h, int prec, const ps_tuning* t) {
  if (!h || h->sph) return fail(PS_ERR_INVALID_ARG, "poisson_set_tuning needs a Cartesian handle");
  if (prec < PS_FP64 || prec > PS_MIXED_BF16) return fail(PS_ERR_INVALID_ARG, "unknown precision %d", prec);
  if (!t) {
    h->has_tun[prec] = 0;
    return PS_OK;
  }
  if (t->nu1 < 0 || t->nu2 < 0 || t->nu1 + t->nu2 < 1 || t->nu1 > 64 || t->nu2 > 64)
    return fail(PS_ERR_INVALID_ARG, "tuning: nu1, nu2 in 0..64 with nu1 + nu2 >= 1");
  if (t->inner_cycles < 1 || t->inner_cycles > 64) return fail(PS_ERR_INVALID_ARG, "tuning: inner_cycles in 1..64");
  if (t->sweep_tile < 0 || t->sweep_tile > kRbSweepTiles)
    return fail(PS_ERR_INVALID_ARG, "tuning: sweep_tile in 0..%d", kRbSweepTiles);
  if (t->restrict_tile < 0 || t->restrict_tile > kRrTiles)
    return fail(PS_ERR_INVALID_ARG, "tuning: restrict_tile in 0..%d", kRrTiles);
  h->tun[prec] = *t;
  h->has_tun[prec] = 1;
  return PS_OK;
}

ps_status poisson_get_tuning(ps_handle h, int prec, ps_tuning* out, int* is_set) {
  if (!h || !out || !is_set) return fail(PS_ERR_INVALID_ARG, "poisson_get_tuning: NULL argument");
  if (prec < PS_FP64 || prec > PS_MIXED_BF16) return fail(PS_ERR_INVALID_ARG, "unknown precision %d", prec);
  *is_set = h->has_tun[prec];
  if (*is_set) *out = h->tun[prec];
  return PS_OK;
}

size_t poisson_workspace_bytes(const ps_grid* grid, int stencil_order, int l_max, int prec) {
  if (!grid) return 0;
  if (grid->kind == PS_GRID_CART_UNIFORM) {
    if (validate_cart(grid, stencil_order) != PS_OK) return 0;
    return cart_bytes(grid, stencil_order, std::max(0, l_max), prec, true);
  }
  if (grid->kind == PS_GRID_SPHERICAL) {
    const size_t n = (size_t)(grid->n[0] + 2) * (grid->n[1] + 2) * (grid->n[2] + 2);
    const size_t vec = prec == PS_FP64 ? 8 : 4;
    // 8 Krylov vectors, the FP64 iterate and its increments, and the
    // (r, theta) tables (diagonal, rJ, the SOR form)
    return n * (8 * vec + 16) + (size_t)grid->n[0] * grid->n[1] * 80;
  }
  return 0;
}

ps_status poisson_create(const ps_grid* grid, const double* const coords_host[3], int stencil_order,
                         const ps_bc* bc, int l_max, ps_handle* out) {
  if (!grid || !out) return fail(PS_ERR_INVALID_ARG, "grid and out must not be NULL");
  *out = nullptr;
  ps_bc b{};
  b.outer = PS_BC_DIRICHLET_GIVEN;
  b.inner = PS_INNER_NONE;
  b.G = 1.0;
  if (bc) b = *bc;
  if (b.outer != PS_BC_DIRICHLET_GIVEN && b.outer != PS_BC_MULTIPOLE)
    return fail(PS_ERR_INVALID_ARG, "unknown outer boundary %d", b.outer);
  if (!std::isfinite(b.G)) return fail(PS_ERR_INVALID_ARG, "G must be finite");
  if (b.outer == PS_BC_MULTIPOLE && (l_max < 0 || l_max > 16))
    return fail(PS_ERR_INVALID_ARG, "l_max must be in 0..16 (got %d)", l_max);
  if (grid->kind == PS_GRID_CART_UNIFORM) {
    ps_status s = validate_cart(grid, stencil_order);
    if (s != PS_OK) return s;
    if (b.inner != PS_INNER_NONE) return fail(PS_ERR_INVALID_ARG, "Cartesian grids take no inner boundary");
  } else if (grid->kind == PS_GRID_SPHERICAL) {
    if (stencil_order != 2) return fail(PS_ERR_INVALID_ARG, "spherical grids use the 7-point operator (order 2)");
    if (!coords_host || !coords_host[0] || !coords_host[1] || !coords_host[2])
      return fail(PS_ERR_INVALID_ARG, "spherical grids need coords r, theta, phi");
    const int nr = grid->n[0], nt = grid->n[1], np = grid->n[2];
    if (nr < 3 || nt < 2 || np < 3) return fail(PS_ERR_INVALID_ARG, "spherical grid too small");
    const double* r = coords_host[0];
    if (!(r[0] > 0.0)) return fail(PS_ERR_INVALID_ARG, "r[0] must be positive");
    for (int i = 1; i < nr; i++)
      if (!(r[i] > r[i - 1])) return fail(PS_ERR_INVALID_ARG, "r must increase");
    for (int j = 0; j < nt; j++) {
      const double want = (j + 0.5) * M_PI / nt;
      if (std::fabs(coords_host[1][j] - want) > 1e-9) return fail(PS_ERR_INVALID_ARG, "theta_j must be (j+1/2) pi / Ntheta");
    }
    for (int k = 0; k < np; k++) {
      const double want = 2.0 * M_PI * k / np;
      if (std::fabs(coords_host[2][k] - want) > 1e-9) return fail(PS_ERR_INVALID_ARG, "phi_k must be 2 pi k / Nphi");
    }
    if (b.inner != PS_INNER_NEUMANN && b.inner != PS_INNER_MULTIPOLE)
      return fail(PS_ERR_UNSUPPORTED, "spherical grids take the Neumann or the multipole inner boundary");
    if (b.inner == PS_INNER_MULTIPOLE && l_max < 0) return fail(PS_ERR_INVALID_ARG, "the multipole inner boundary needs l_max >= 0");
  } else {
    return fail(PS_ERR_INVALID_ARG, "unknown grid kind %d", grid->kind);
  }

  ps_ctx* h = new ps_ctx();
  h->grid = *grid;
  h->order = stencil_order;
  h->bc = b;
  h->lmax = l_max;
  h->sph = grid->kind == PS_GRID_SPHERICAL;
  auto bail = [&](ps_status s) {
    poisson_destroy(h);
    return s;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(fail(PS_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
  if ((e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(fail(PS_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
  for (auto& ev : h->ev)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(fail(PS_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e)));
  if ((e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming)) != cudaSuccess)
    return bail(fail(PS_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e)));
  if ((e = cudaMalloc(&h->st, sizeof(DevState))) != cudaSuccess) return bail(fail(PS_ERR_OOM, "state alloc"));
  if ((e = cudaMallocHost(&h->hst, sizeof(DevState))) != cudaSuccess) return bail(fail(PS_ERR_OOM, "pinned alloc"));
  memset(h->hst, 0, sizeof(DevState));
  h->st_active = h->st;
  ps_status s;
  if (!h->sph) {
    const int gw = stencil_order / 2;
    std::vector<std::array<int, 3>> lv;
    levels_for(grid->n, &lv);
    h->nlev = (int)lv.size();
    for (int l = 0; l < h->nlev; l++) {
      h->dims.push_back(level_dims(lv[l], gw, l + 1 == h->nlev));
      std::array<double, 3> hh;
      for (int a = 0; a < 3; a++) hh[a] = (grid->hi[a] - grid->lo[a]) / lv[l][a];
      h->hs.push_back(hh);
    }
    h->d0 = h->dims[0];
    h->du = make_dims(grid->n[0], grid->n[1], grid->n[2], gw);
    for (int a = 0; a < 3; a++) h->h0[a] = h->hs[0][a];
    if ((s = alloc_zero((void**)&h->fs64, (size_t)h->d0.size() * 8, &h->bytes)) != PS_OK) return bail(s);
    if ((s = alloc_zero((void**)&h->phi0, (size_t)h->d0.size() * 8, &h->bytes)) != PS_OK) return bail(s);
    if ((s = ensure_partials(h, std::max({cart_partials_count(h->d0), delta_colours_partials(h->d0, stencil_order),
                                                  batch_norm_partials(h->d0, stencil_order),
                                                  stencil_order == 2 ? 2 * c27_blocks(h->d0) : 0}))) != PS_OK)
      return bail(s);
    if (b.outer == PS_BC_MULTIPOLE) {
      build_multipole_tables(l_max, &h->mpt);
      if ((e = cart_multipole_alloc(h->du, l_max, h->mpt, &h->mp)) != cudaSuccess)
        return bail(fail(PS_ERR_OOM, "multipole alloc: %s", cudaGetErrorString(e)));
      h->bytes += h->mp.bytes;
    }
    // the coarsest level must fit one CTA's shared memory for the coarse CG
    const Dims& dc = h->dims.back();
    if (h->nlev >= 2 && coarse_cg_smem_bytes(dc) > 200 * 1024)
      return bail(fail(PS_ERR_INVALID_ARG, "coarsest level %dx%dx%d too large for the single-CTA CG", dc.nx, dc.ny, dc.nz));
  } else {
    h->sd.nr = grid->n[0];
    h->sd.nt = grid->n[1];
    h->sd.np = grid->n[2];
    const bool inner_mp = b.inner == PS_INNER_MULTIPOLE;
    h->sd.inner_ghost = inner_mp ? 1 : 0;
    if (inner_mp && !(2.0 * coords_host[0][0] - coords_host[0][1] > 0.0))
      return bail(fail(PS_ERR_INVALID_ARG, "the multipole inner boundary needs the ghost radius 2 r_0 - r_1 > 0"));
    if ((e = sph_tables_build(h->sd, coords_host[0], coords_host[1], coords_host[2],
                              b.outer == PS_BC_MULTIPOLE || inner_mp ? l_max : -1, &h->stab, inner_mp)) != cudaSuccess)
      return bail(fail(PS_ERR_OOM, "spherical tables: %s", cudaGetErrorString(e)));
    h->bytes += h->stab.bytes;
    if ((s = alloc_zero((void**)&h->phi0, (size_t)h->sd.size() * 8, &h->bytes)) != PS_OK) return bail(s);
    const int nblk = ((h->sd.nr + 31) / 32) * ((h->sd.nt + 7) / 8) * h->sd.np;
    if ((s = ensure_partials(h, nblk)) != PS_OK) return bail(s);
  }
  *out = h;
  return PS_OK;
}

void poisson_destroy(ps_handle h) {
  if (!h) return;
  drop_graphs(h);
  cudaFree(h->phi0);
  if (h->cap) cudaStreamDestroy(h->cap);
  free_hier(&h->h64);
  free_hier(&h->hmx[0]);
  free_hier(&h->hmx[1]);
  cudaFree(h->fs64);
  cudaFree(h->cg_r);
  cudaFree(h->cg_p);
  cudaFree(h->cg_q);
  cudaFree(h->cg_z);
  cudaFree(h->sph_w);
  cudaFree(h->sph_g);
  cudaFree(h->sor_wtab);
  cart_multipole_free(&h->mp);
  sph_tables_free(&h->stab);
  for (auto& p : h->sv) cudaFree(p);
  cudaFree(h->sz);
  cudaFree(h->partials);
  cudaFree(h->st);
  if (h->hst) cudaFreeHost(h->hst);
  for (auto& ev : h->ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& r : h->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto ev : h->ev_pool) cudaEventDestroy(ev);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

ps_status poisson_solve_begin(ps_handle h, const double* rho_dev, double* phi_dev, double tol,
                              const ps_solve_opts* opts) {
  if (!h) return fail(PS_ERR_INVALID_ARG, "NULL handle");
  if (h->act.on) return fail(PS_ERR_INVALID_ARG, "a solve is already in flight on this handle");
  if (!rho_dev || !phi_dev) return fail(PS_ERR_INVALID_ARG, "rho and phi must be device pointers");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(PS_ERR_INVALID_ARG, "tol must be finite and >= 0");
  ps_solve_opts o{};
  o.method = PS_MG;
  o.prec = PS_FP64;
  o.omega = 1.0;
  o.nu1 = 2;
  o.nu2 = 2;
  o.max_iter = 100;
  o.inner_cycles = 1;
  if (opts) o = *opts;
  if (o.max_iter < 0) return fail(PS_ERR_INVALID_ARG, "max_iter must be >= 0");
  if (o.prec < PS_FP64 || o.prec > PS_MIXED_BF16) return fail(PS_ERR_INVALID_ARG, "unknown precision %d", o.prec);
  int sweep_tile = 0, restrict_tile = 0;
  if (o.use_tuning && !h->sph && o.method == PS_MG && h->has_tun[o.prec]) {
    const ps_tuning& t = h->tun[o.prec];
    o.nu1 = t.nu1;
    o.nu2 = t.nu2;
    o.inner_cycles = t.inner_cycles;
    o.tile_min_n = t.tile_min_n;
    sweep_tile = t.sweep_tile;
    restrict_tile = t.restrict_tile;
  }
  if (o.sor_schedule < PS_SOR_FIXED || o.sor_schedule > PS_SOR_OPTIMAL)
    return fail(PS_ERR_INVALID_ARG, "unknown SOR schedule %d", o.sor_schedule);
  if (o.method == PS_SOR && o.sor_schedule == PS_SOR_FIXED && !(o.omega > 0.0 && o.omega < 2.0))
    return fail(PS_ERR_INVALID_ARG, "SOR needs 0 < omega < 2");
  if (h->sph) {
    if (o.method != PS_BICGSTAB && o.method != PS_SOR)
      return fail(PS_ERR_UNSUPPORTED, "spherical grids are solved by BiCGSTAB or SOR (method %d)", o.method);
    if (o.method == PS_SOR && o.prec != PS_FP64) return fail(PS_ERR_UNSUPPORTED, "SOR runs in FP64 only");
    if (o.prec == PS_MIXED_BF16) return fail(PS_ERR_UNSUPPORTED, "BF16 storage is a multigrid option");
  } else if (o.method == PS_MG) {
    if (h->nlev < 2) return fail(PS_ERR_INVALID_ARG, "multigrid needs all interval counts even and >= 16");
    if (o.nu1 < 0 || o.nu2 < 0 || o.nu1 + o.nu2 < 1) return fail(PS_ERR_INVALID_ARG, "nu1, nu2 >= 0 with nu1 + nu2 >= 1");
    if (o.compact_order != 0) {
      if (o.compact_order != 2 && o.compact_order != 4 && o.compact_order != 6)
        return fail(PS_ERR_INVALID_ARG, "compact_order must be 0, 2, 4 or 6 (got %d)", o.compact_order);
      if (h->order != 2) return fail(PS_ERR_INVALID_ARG, "compact stencils need a handle created with stencil_order 2 (radius-one layout)");
      if (o.prec == PS_MIXED_BF16) return fail(PS_ERR_UNSUPPORTED, "the compact-stencil multigrid runs in FP64 or with FP32 refinement");
      if (!(std::fabs(h->h0[0] - h->h0[1]) <= 1e-14 * h->h0[0] && std::fabs(h->h0[1] - h->h0[2]) <= 1e-14 * h->h0[0]))
        return fail(PS_ERR_INVALID_ARG, "compact stencils and SPAI smoothers need equal spacings on every axis");
      if (c27_coarse_smem(h->dims.back()) > 200 * 1024) return fail(PS_ERR_INVALID_ARG, "coarsest level too large for the compact coarse CG");
    }
  } else if (o.method == PS_SOR) {
    if (o.prec != PS_FP64) return fail(PS_ERR_UNSUPPORTED, "SOR runs in FP64 only");
  } else if (o.method == PS_CG || o.method == PS_PCG) {
    if (o.prec != PS_FP64) return fail(PS_ERR_UNSUPPORTED, "CG runs in FP64 only");
  } else {
    return fail(PS_ERR_INVALID_ARG, "method %d is not available on Cartesian grids", o.method);
  }
  Active& a = h->act;
  a = Active();
  a.o = o;
  a.sweep_tile = sweep_tile;
  a.restrict_tile = restrict_tile;
  a.tol = tol;
  a.rho = rho_dev;
  a.phi_user = phi_dev;
  a.caller = (cudaStream_t)o.stream;   // NULL = CUDA's default stream
  h->nlaunch = 0;
  // the handle's stream starts after everything the caller enqueued so far
  cudaStream_t s = h->stream;
  TRY(cudaEventRecord(h->ev_in, a.caller));
  TRY(cudaStreamWaitEvent(s, h->ev_in, 0));
  ps_status r;
  if (h->sph) {
    r = begin_sph(h, rho_dev, phi_dev, tol, &o, s);
  } else {
    const bool compact = o.method == PS_MG && o.compact_order != 0;
    if ((r = cart_prepare(h, rho_dev, phi_dev, tol, o.max_iter, compact, s)) != PS_OK) return r;
    if (o.method == PS_MG && o.compact_order != 0)
      r = o.prec == PS_FP64 ? begin_mg_compact(h, rho_dev, &o, s) : begin_ir_compact(h, rho_dev, &o, s);
    else if (o.method == PS_MG) r = o.prec == PS_FP64 ? begin_mg64(h, &o, s) : begin_ir(h, &o, s);
    else if (o.method == PS_SOR) r = begin_sor(h, &o, s);
    else if (o.method == PS_PCG) r = begin_pcg(h, s);
    else r = begin_cg(h, s);
  }
  if (r != PS_OK) return r;
  h->hst->iter = 0;
  h->hst->done = DONE_NO;
  a.on = true;
  return PS_OK;
}

ps_status poisson_solve_step(ps_handle h, int max_iterations) {
  if (!h || !h->act.on) return fail(PS_ERR_INVALID_ARG, "no solve in flight");
  if (max_iterations < 1) return fail(PS_ERR_INVALID_ARG, "max_iterations must be >= 1");
  return step_active(h, max_iterations);
}

ps_status poisson_solve_poll(ps_handle h, int* done, ps_info* info) {
  if (!h || !h->act.on || !done) return fail(PS_ERR_INVALID_ARG, "no solve in flight / NULL done");
  ps_status r = poll_active(h, done);
  if (r != PS_OK) return r;
  if (info) fill_info(h, info, PS_OK, false);
  return PS_OK;
}

ps_status poisson_solve_end(ps_handle h, ps_info* info) {
  if (!h || !h->act.on) return fail(PS_ERR_INVALID_ARG, "no solve in flight");
  Active& a = h->act;
  cudaStream_t s = h->stream;
  a.on = false;
  TRY(cudaEventRecord(h->ev[2], s));
  if (h->sph) TRY(cudaMemcpyAsync(a.phi_user, h->phi0, (size_t)h->sd.size() * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else TRY(copy_rows(a.phi_user, h->du, h->phi0, h->d0, s));
  TRY(cudaEventRecord(h->ev_out, s));
  TRY(cudaStreamWaitEvent(a.caller, h->ev_out, 0));
  int done = 0;
  ps_status r = poll_active(h, &done);
  if (r != PS_OK) return r;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PS_ERR_CUDA, "solve: %s", cudaGetErrorString(e));
  ps_status out = PS_OK;
  if (h->hst->done == DONE_MAXITER || h->hst->done == DONE_NO) out = PS_NOT_CONVERGED;
  else if (h->hst->done == DONE_DIVERGED) out = PS_DIVERGED;
  else if (h->hst->done == DONE_FAULT) return fail(PS_ERR_TIMEOUT, "a tile kernel's TMA copy did not complete; the result is invalid");
  if (out == PS_NOT_CONVERGED) fail(out, "not converged: relative residual %.3e after %d iterations", h->hst->rel, h->hst->iter);
  if (out == PS_DIVERGED) fail(out, "diverged: relative residual %.3e after %d iterations", h->hst->rel, h->hst->iter);
  fill_info(h, info, out, true);
  return out;
}

ps_status poisson_solve(ps_handle h, const double* rho_dev, double* phi_dev, double tol,
                        const ps_solve_opts* opts, ps_info* info) {
  ps_status r = poisson_solve_begin(h, rho_dev, phi_dev, tol, opts);
  if (r != PS_OK) return r;
  int done = 0;
  if ((r = poll_active(h, &done)) != PS_OK) { h->act.on = false; return r; }
  while (!done) {
    if ((r = step_active(h, h->act.chunk)) != PS_OK || (r = poll_active(h, &done)) != PS_OK) {
      h->act.on = false;
      return r;
    }
  }
  return poisson_solve_end(h, info);
}

// Batched solve: every request runs on its own handle's stream, so their kernels
// overlap on the GPU; each request's kernels and reductions are exactly those
// of a solo solve, so results equal separate poisson_solve calls bit for bit.
ps_status poisson_solve_batch(ps_handle* hs, const double* const* rho, double* const* phi,
                              const double* tol, int n, const ps_solve_opts* opts, ps_info* infos) {
  if (n < 0 || (n > 0 && (!hs || !rho || !phi || !tol))) return fail(PS_ERR_INVALID_ARG, "bad batch arguments");
  for (int i = 0; i < n; i++) {
    if (!hs[i]) return fail(PS_ERR_INVALID_ARG, "NULL handle in batch");
    for (int j = i + 1; j < n; j++)
      if (hs[i] == hs[j]) return fail(PS_ERR_INVALID_ARG, "batch handles must be distinct");
  }
  ps_status r;
  std::vector<int> done(n, 0);
  for (int i = 0; i < n; i++)
    if ((r = poisson_solve_begin(hs[i], rho[i], phi[i], tol[i], opts)) != PS_OK) {
      for (int j = 0; j < i; j++) hs[j]->act.on = false;
      return r;
    }
  int left = n;
  for (int i = 0; i < n; i++) {
    if ((r = poll_active(hs[i], &done[i])) != PS_OK) return r;
    if (done[i]) left--;
  }
  while (left > 0) {
    for (int i = 0; i < n; i++)
      if (!done[i] && (r = step_active(hs[i], hs[i]->act.chunk)) != PS_OK) return r;
    for (int i = 0; i < n; i++) {
      if (done[i]) continue;
      if ((r = poll_active(hs[i], &done[i])) != PS_OK) return r;
      if (done[i]) left--;
    }
  }
  ps_status worst = PS_OK;
  for (int i = 0; i < n; i++) {
    ps_status si = poisson_solve_end(hs[i], infos ? &infos[i] : nullptr);
    if (si != PS_OK && si != PS_NOT_CONVERGED && si != PS_DIVERGED) return si;
    if (si != PS_OK && worst == PS_OK) worst = si;
  }
  return worst;
}


// ---------------------------------------------------------------------- batched executor
ps_status poisson_batch_create(int capacity, int max_n, int stencil_order, int prec, int nu1, int nu2,
                               int inner_cycles, ps_batch* out) {
  if (!out) return fail(PS_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  if (capacity < 1 || capacity > 1024) return fail(PS_ERR_INVALID_ARG, "capacity must be in 1..1024 (got %d)", capacity);
  if (stencil_order != 2 && stencil_order != 4) return fail(PS_ERR_INVALID_ARG, "stencil_order must be 2 or 4");
  if (prec != PS_FP64 && prec != PS_MIXED_FP32)
    return fail(PS_ERR_UNSUPPORTED, "batches run in FP64 or with FP32 refinement (precision %d)", prec);
  if (nu1 < 1 || nu2 < 0) return fail(PS_ERR_INVALID_ARG, "batches need nu1 >= 1 and nu2 >= 0");
  if (prec == PS_MIXED_FP32 && inner_cycles < 1) return fail(PS_ERR_INVALID_ARG, "inner_cycles must be >= 1");
  const int nmax[3] = {max_n, max_n, max_n};
  std::vector<std::array<int, 3>> lv;
  if (max_n < 16 || max_n > 8192) return fail(PS_ERR_INVALID_ARG, "max_n must be in 16..8192");
  levels_for(nmax, &lv);
  int nlev_max = (int)lv.size();
  // a grid no larger than max_n on every axis has at most this many levels
  for (int n = 16; n <= max_n; n++) {
    const int nn[3] = {n, n, n};
    levels_for(nn, &lv);
    nlev_max = std::max(nlev_max, (int)lv.size());
  }
  if (nlev_max > PS_BMAX_LEVELS) return fail(PS_ERR_INVALID_ARG, "max_n too large for a batch");
  ps_batch_ctx* b = new ps_batch_ctx();
  b->cap = capacity;
  b->order = stencil_order;
  b->prec = prec;
  b->nu1 = nu1;
  b->nu2 = nu2;
  b->inner = prec == PS_FP64 ? 1 : inner_cycles;
  b->nlev_max = nlev_max;
  b->slots.resize(capacity);
  b->hslots.assign(capacity, BSlot());
  for (auto& sd : b->hslots) memset(&sd, 0, sizeof(sd));
  b->kernels_per_iter = batch_kernels_per_iteration(nlev_max, stencil_order, prec == PS_FP64 ? 0 : 1, nu1, nu2, b->inner);
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&b->capstream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaMalloc(&b->dslots, (size_t)capacity * sizeof(BSlot))) != cudaSuccess ||
      (e = cudaMalloc(&b->dlists, (size_t)BL_NKINDS * PS_BMAX_LEVELS * sizeof(BList))) != cudaSuccess ||
      (e = cudaMalloc(&b->dstatus, (size_t)capacity * 2 * sizeof(int))) != cudaSuccess ||
      (e = cudaMallocHost(&b->hstatus, (size_t)capacity * 2 * sizeof(int))) != cudaSuccess) {
    poisson_batch_destroy(b);
    return fail(e == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA, "batch allocation: %s", cudaGetErrorString(e));
  }
  *out = b;
  return PS_OK;
}

void poisson_batch_destroy(ps_batch b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  destroy_batch_graphs(b);
  for (auto& sl : b->slots)
    if (sl.h) sl.h->in_batch = false;
  cudaFree(b->dslots);
  cudaFree(b->ditems);
  cudaFree(b->dlists);
  cudaFree(b->dstatus);
  if (b->hstatus) cudaFreeHost(b->hstatus);
  if (b->capstream) cudaStreamDestroy(b->capstream);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

ps_status poisson_batch_add(ps_batch b, ps_handle h, const double* rho_dev, double* phi_dev, double tol,
                            int max_iter, int* slot) {
  if (!b || !h || !slot) return fail(PS_ERR_INVALID_ARG, "NULL batch, handle or slot");
  *slot = -1;
  if (!rho_dev || !phi_dev) return fail(PS_ERR_INVALID_ARG, "rho and phi must be device pointers");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(PS_ERR_INVALID_ARG, "tol must be finite and >= 0");
  if (max_iter < 0) return fail(PS_ERR_INVALID_ARG, "max_iter must be >= 0");
  if (h->sph) return fail(PS_ERR_UNSUPPORTED, "batches hold Cartesian multigrid solves");
  if (h->order != b->order) return fail(PS_ERR_INVALID_ARG, "the handle's stencil order differs from the batch's");
  if (h->nlev < 2) return fail(PS_ERR_INVALID_ARG, "multigrid needs all interval counts even and >= 16");
  if (h->nlev > b->nlev_max) return fail(PS_ERR_INVALID_ARG, "grid larger than the batch's max_n");
  if (h->act.on || h->in_batch) return fail(PS_ERR_INVALID_ARG, "the handle has a solve in flight");
  const Dims& dc = h->dims.back();
  if ((long long)dc.ni() * dc.nj() * dc.nk() > 16 * 256)
    return fail(PS_ERR_UNSUPPORTED, "coarsest level too large for the batched coarsest CG (at most 4096 unknowns)");
  int si = -1;
  for (int i = 0; i < b->cap; i++)
    if (!b->hslots[i].active) { si = i; break; }
  if (si < 0) return fail(PS_ERR_INVALID_ARG, "the batch is full");
  cudaStream_t s = b->stream;
  // start after everything the caller enqueued on CUDA's default stream
  TRY(cudaEventRecord(h->ev_in, 0));
  TRY(cudaStreamWaitEvent(s, h->ev_in, 0));
  h->nlaunch = 0;
  ps_status r;
  if ((r = cart_prepare(h, rho_dev, phi_dev, tol, max_iter, false, s)) != PS_OK) return r;
  Hier* H = b->prec == PS_FP64 ? &h->h64 : &h->hmx[0];
  if ((r = build_hier(h, b->prec == PS_FP64 ? 0 : 1, H)) != PS_OK) return r;
  if (b->prec == PS_FP64) {
    H->lv[0].phi = h->phi0;
    TRY(norm_pass(h, h->phi0, 1, DT_F64, nullptr, s, 0, 0, false, true));
  } else {
    TRY(norm_pass(h, h->phi0, 1, H->lv[0].dt, H->lv[0].fs, s, 0, 0, false, true));
  }
  BSlot& sd = b->hslots[si];
  memset(&sd, 0, sizeof(sd));
  for (int l = 0; l < h->nlev; l++) batch_level_desc(h, H->lv[l], &sd.lv[l]);
  sd.st = h->st;
  sd.phi64 = h->phi0;
  sd.fs64 = h->fs64;
  sd.cf0 = make_coef<double>(h->d0, h->h0, h->order);
  sd.dscale = sd.cf0.d;
  sd.nlev = h->nlev;
  sd.active = 1;
  b->slots[si].h = h;
  b->slots[si].phi_user = phi_dev;
  h->in_batch = true;
  h->act = Active();
  h->act.inner_per_iter = b->prec == PS_FP64 ? 0 : b->inner;
  h->hst->iter = 0;
  h->hst->done = DONE_NO;
  b->dirty = true;
  *slot = si;
  return PS_OK;
}

ps_status poisson_batch_step(ps_batch b, int iterations) {
  if (!b) return fail(PS_ERR_INVALID_ARG, "NULL batch");
  if (iterations < 1 || iterations > 64) return fail(PS_ERR_INVALID_ARG, "iterations must be in 1..64");
  ps_status r;
  if (b->dirty && (r = batch_rebuild(b)) != PS_OK) return r;
  cudaGraphExec_t g = nullptr;
  if ((r = batch_graph(b, iterations, &g)) != PS_OK) return r;
  TRY(cudaGraphLaunch(g, b->stream));
  for (int i = 0; i < b->cap; i++)
    if (b->hslots[i].active) b->slots[i].h->nlaunch += (long long)b->kernels_per_iter * iterations;
  return PS_OK;
}

ps_status poisson_batch_poll(ps_batch b, int32_t* status, int32_t* iterations) {
  if (!b || !status) return fail(PS_ERR_INVALID_ARG, "NULL batch or status");
  if (b->dirty) {
    ps_status r = batch_rebuild(b);
    if (r != PS_OK) return r;
  }
  TRY(launch_b_gather(b->dslots, b->cap, b->dstatus, b->stream));
  TRY(cudaMemcpyAsync(b->hstatus, b->dstatus, (size_t)b->cap * 2 * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  TRY(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < b->cap; i++) {
    status[i] = b->hstatus[2 * i];
    if (iterations) iterations[i] = b->hstatus[2 * i + 1];
  }
  return PS_OK;
}

ps_status poisson_batch_remove(ps_batch b, int slot, ps_info* info) {
  if (!b || slot < 0 || slot >= b->cap || !b->hslots[slot].active)
    return fail(PS_ERR_INVALID_ARG, "no solve in batch slot %d", slot);
  ps_ctx* h = b->slots[slot].h;
  cudaStream_t s = b->stream;
  TRY(cudaEventRecord(h->ev[2], s));
  TRY(copy_rows(b->slots[slot].phi_user, h->du, h->phi0, h->d0, s));
  TRY(cudaEventRecord(h->ev_out, s));
  TRY(cudaStreamWaitEvent(0, h->ev_out, 0));
  ps_status r = read_state(h, s);
  b->hslots[slot].active = 0;
  b->slots[slot] = BSlotHost();
  h->in_batch = false;
  b->dirty = true;
  if (r != PS_OK) return r;
  ps_status out = PS_OK;
  if (h->hst->done == DONE_MAXITER || h->hst->done == DONE_NO) out = PS_NOT_CONVERGED;
  else if (h->hst->done == DONE_DIVERGED) out = PS_DIVERGED;
  else if (h->hst->done == DONE_FAULT) return fail(PS_ERR_TIMEOUT, "a kernel's wait did not complete; the result is invalid");
  fill_info(h, info, out, true);
  return out;
}

ps_status poisson_profile_enable(ps_handle h, int enable) {
  if (!h) return fail(PS_ERR_INVALID_ARG, "NULL handle");
  h->prof = enable != 0;
  return PS_OK;
}

int poisson_profile_read(ps_handle h, ps_kernel_stat* out, int max) {
  if (!h || (max > 0 && !out)) {
    fail(PS_ERR_INVALID_ARG, "bad profile_read arguments");
    return -1;
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    fail(PS_ERR_CUDA, "profile_read: synchronisation failed");
    return -1;
  }
  struct Acc { int64_t n = 0; double ms = 0, bytes = 0, ops = 0; int fp64 = 0, variant = 0; };
  std::vector<Acc> acc(PC_COUNT);
  for (int c = 0; c < PC_COUNT; c++) {
    acc[c].n = h->acc[c].n;
    acc[c].ms = h->acc[c].ms;
    acc[c].bytes = h->acc[c].bytes;
    acc[c].ops = h->acc[c].ops;
    acc[c].fp64 = h->acc[c].fp64;
    acc[c].variant = h->acc[c].variant;
    h->acc[c] = ProfAcc();
  }
  for (auto& r : h->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      Acc& a = acc[r.cls];
      a.n++;
      a.ms += ms;
      a.bytes += r.bytes;
      a.ops += r.ops;
      a.fp64 = r.fp64;
      a.variant = r.variant;
    }
    h->ev_pool.push_back(r.a);
    h->ev_pool.push_back(r.b);
  }
  h->recs.clear();
  int k = 0;
  for (int c = 0; c < PC_COUNT; c++) {
    if (acc[c].n == 0) continue;
    if (k < max) {
      ps_kernel_stat& o = out[k];
      memset(&o, 0, sizeof(o));
      snprintf(o.name, sizeof(o.name), "%s", kProfNames[c]);
      o.launches = acc[c].n;
      o.total_ms = acc[c].ms;
      // a class can mix launches of different work (a full residual and a
      // one-colour residual are both convergence passes): report the mean
      o.bytes_per_launch = acc[c].bytes / (double)acc[c].n;
      o.ops_per_launch = acc[c].ops / (double)acc[c].n;
      o.fp64 = acc[c].fp64;
      o.variant = acc[c].variant;
    }
    k++;
  }
  return k;
}

// ---------------------------------------------------------------------- op-level calls
static ps_status op_dims(const ps_grid* g, int order, int dtype, Dims* d, double h[3]) {
  if (!g || g->kind != PS_GRID_CART_UNIFORM) return fail(PS_ERR_INVALID_ARG, "Cartesian grid required");
  ps_status s = validate_cart(g, order);
  if (s != PS_OK) return s;
  if (dtype < 0 || dtype > 2) return fail(PS_ERR_INVALID_ARG, "dtype must be 0, 1 or 2");
  *d = make_dims(g->n[0], g->n[1], g->n[2], order / 2);
  for (int a = 0; a < 3; a++) h[a] = (g->hi[a] - g->lo[a]) / g->n[a];
  return PS_OK;
}

ps_status ps_op_apply(const ps_grid* grid, int order, int dtype, const void* phi, void* out, void* stream) {
  Dims d;
  double h[3];
  ps_status s = op_dims(grid, order, dtype, &d, h);
  if (s != PS_OK) return s;
  if (!phi || !out) return fail(PS_ERR_INVALID_ARG, "NULL buffer");
  TRY(launch_apply(d, order, h, dtype, phi, out, (cudaStream_t)stream));
  return PS_OK;
}

ps_status ps_op_residual(const ps_grid* grid, int order, int dtype, const void* phi, const void* f,
                         void* r, double* norm2_host, void* stream) {
  Dims d;
  double h[3];
  ps_status s = op_dims(grid, order, dtype, &d, h);
  if (s != PS_OK) return s;
  if (!phi || !f || !r) return fail(PS_ERR_INVALID_ARG, "NULL buffer");
  cudaStream_t st = (cudaStream_t)stream;
  // r = f - A phi through the scaled form: fs = -f/d, delta = phi_GS - phi, r = -d delta
  Coef<double> cf = make_coef<double>(d, h, order);
  const size_t esz = dt_size(dtype);
  void* fs = nullptr;
  double* part = nullptr;
  const int nb = cart_partials_count(d);
  TRY(cudaMalloc(&fs, (size_t)d.size() * esz));
  TRY(cudaMalloc(&part, (size_t)nb * 2 * sizeof(double)));
  cudaError_t e = cudaMemsetAsync(fs, 0, (size_t)d.size() * esz, st);
  // scale f into fs by a delta pass of a zero field: reuse the apply path
  if (e == cudaSuccess) e = launch_scale_rhs_any(d, -cf.inv_d, dtype, f, fs, st);
  if (e == cudaSuccess) e = launch_delta(d, order, h, dtype, phi, fs, dtype, r, -cf.d, false, part, nullptr, st);
  double S = 0.0;
  if (e == cudaSuccess && norm2_host) {
    std::vector<double> hp((size_t)nb * 2);
    e = cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int b = 0; b < nb; b++) S += hp[2 * b];
    *norm2_host = S * cf.d * cf.d;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(fs);
  cudaFree(part);
  if (e != cudaSuccess) return fail(PS_ERR_CUDA, "ps_op_residual: %s", cudaGetErrorString(e));
  return PS_OK;
}

ps_status ps_op_sweep(const ps_grid* grid, int order, int dtype, void* phi, const void* f, double omega,
                      void* stream) {
  Dims d;
  double h[3];
  ps_status s = op_dims(grid, order, dtype, &d, h);
  if (s != PS_OK) return s;
  if (!phi || !f) return fail(PS_ERR_INVALID_ARG, "NULL buffer");
  if (!(omega > 0.0 && omega < 2.0)) return fail(PS_ERR_INVALID_ARG, "0 < omega < 2 required");
  cudaStream_t st = (cudaStream_t)stream;
  Coef<double> cf = make_coef<double>(d, h, order);
  void* fs = nullptr;
  TRY(cudaMalloc(&fs, (size_t)d.size() * dt_size(dtype)));
  cudaError_t e = launch_scale_rhs_any(d, -cf.inv_d, dtype, f, fs, st);
  const int ncol = order == 2 ? 2 : 3;
  for (int c = 0; c < ncol && e == cudaSuccess; c++)
    e = launch_sweep_colour(d, order, h, dtype, phi, fs, c, omega, nullptr, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(fs);
  if (e != cudaSuccess) return fail(PS_ERR_CUDA, "ps_op_sweep: %s", cudaGetErrorString(e));
  return PS_OK;
}

ps_status ps_op_restrict(const ps_grid* grid, int order, int dtype, const void* rf, void* fc, void* stream) {
  Dims d;
  double h[3];
  ps_status s = op_dims(grid, order, dtype, &d, h);
  if (s != PS_OK) return s;
  if (d.nx % 2 || d.ny % 2 || d.nz % 2 || d.nx < 4 || d.ny < 4 || d.nz < 4)
    return fail(PS_ERR_INVALID_ARG, "restriction needs even interval counts >= 4");
  if (dtype == DT_BF16) return fail(PS_ERR_UNSUPPORTED, "coarse levels are FP32 or FP64");
  TRY(launch_restrict(d, make_dims(d.nx / 2, d.ny / 2, d.nz / 2, d.g), dtype, rf, dtype, fc, 1.0, (cudaStream_t)stream));
  return PS_OK;
}

ps_status ps_op_restrict_red(const ps_grid* grid, int order, int dtype, const void* rf, void* fc, void* stream) {
  Dims d;
  double h[3];
  ps_status s = op_dims(grid, order, dtype, &d, h);
  if (s != PS_OK) return s;
  if (order != 2) return fail(PS_ERR_INVALID_ARG, "the red-only restriction is for the 7-point stencil");
  if (d.nx % 2 || d.ny % 2 || d.nz % 2 || d.nx < 4 || d.ny < 4 || d.nz < 4)
    return fail(PS_ERR_INVALID_ARG, "restriction needs even interval counts >= 4");
  if (dtype == DT_BF16) return fail(PS_ERR_UNSUPPORTED, "coarse levels are FP32 or FP64");
  TRY(launch_restrict_red(d, make_dims(d.nx / 2, d.ny / 2, d.nz / 2, d.g), dtype, rf, dtype, fc, 1.0,
                          (cudaStream_t)stream));
  return PS_OK;
}

ps_status ps_op_prolong(const ps_grid* grid, int order, int dtype, const void* ec, void* phif, void* stream) {
  Dims d;
  double h[3];
  ps_status s = op_dims(grid, order, dtype, &d, h);
  if (s != PS_OK) return s;
  if (d.nx % 2 || d.ny % 2 || d.nz % 2 || d.nx < 4 || d.ny < 4 || d.nz < 4)
    return fail(PS_ERR_INVALID_ARG, "prolongation needs even interval counts >= 4");
  if (dtype == DT_BF16) return fail(PS_ERR_UNSUPPORTED, "coarse levels are FP32 or FP64");
  TRY(launch_prolong(d, make_dims(d.nx / 2, d.ny / 2, d.nz / 2, d.g), dtype, ec, dtype, phif, (cudaStream_t)stream));
  return PS_OK;
}

ps_status ps_op_scale_to_fp32(const double* x, int64_t n, int e, float* out, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return fail(PS_ERR_INVALID_ARG, "NULL buffer or negative n");
  if (e < -100 || e > 100) return fail(PS_ERR_INVALID_ARG, "e must be in -100..100 (got %d)", e);
  TRY(launch_pow2_to_f32(x, (long long)n, e, out, (cudaStream_t)stream));
  return PS_OK;
}

ps_status ps_op_add_scaled_fp32(const float* e, int64_t n, int p, double* phi, void* stream) {
  if (n < 0 || (n > 0 && (!e || !phi))) return fail(PS_ERR_INVALID_ARG, "NULL buffer or negative n");
  if (p < -100 || p > 100) return fail(PS_ERR_INVALID_ARG, "p must be in -100..100 (got %d)", p);
  TRY(launch_add_pow2_f32(e, (long long)n, p, phi, (cudaStream_t)stream));
  return PS_OK;
}

ps_status ps_op_multipole_moments(const ps_grid* grid, int order, const double* rho, const double origin[3],
                                  int l_max, double* q_host, void* stream) {
  Dims d;
  double h[3];
  ps_status s = op_dims(grid, order, 0, &d, h);
  if (s != PS_OK) return s;
  if (l_max < 0 || l_max > 16) return fail(PS_ERR_INVALID_ARG, "l_max must be in 0..16");
  if (!rho || !origin || !q_host) return fail(PS_ERR_INVALID_ARG, "NULL argument");
  MultipoleTables t;
  build_multipole_tables(l_max, &t);
  CartMultipoleDev m;
  cudaError_t e = cart_multipole_alloc(d, l_max, t, &m);
  cudaStream_t st = (cudaStream_t)stream;
  if (e == cudaSuccess) e = launch_cart_moments(d, grid->lo, h, origin, rho, &m, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(q_host, m.q, (size_t)(l_max + 1) * (l_max + 1) * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cart_multipole_free(&m);
  if (e != cudaSuccess) return fail(PS_ERR_CUDA, "ps_op_multipole_moments: %s", cudaGetErrorString(e));
  return PS_OK;
}

ps_status ps_op_multipole_boundary(const ps_grid* grid, int order, const double* q_host, const double origin[3],
                                   int l_max, double G, double* phi, void* stream) {
  Dims d;
  double h[3];
  ps_status s = op_dims(grid, order, 0, &d, h);
  if (s != PS_OK) return s;
  if (l_max < 0 || l_max > 16) return fail(PS_ERR_INVALID_ARG, "l_max must be in 0..16");
  if (!q_host || !origin || !phi) return fail(PS_ERR_INVALID_ARG, "NULL argument");
  MultipoleTables t;
  build_multipole_tables(l_max, &t);
  CartMultipoleDev m;
  cudaError_t e = cart_multipole_alloc(d, l_max, t, &m);
  cudaStream_t st = (cudaStream_t)stream;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m.q, q_host, (size_t)(l_max + 1) * (l_max + 1) * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_cart_faces(d, grid->lo, h, origin, G, m.q, &m, phi, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cart_multipole_free(&m);
  if (e != cudaSuccess) return fail(PS_ERR_CUDA, "ps_op_multipole_boundary: %s", cudaGetErrorString(e));
  return PS_OK;
}

ps_status ps_op_spherical_apply(ps_handle h, const double* phi, double* out, void* stream) {
  if (!h || !h->sph) return fail(PS_ERR_INVALID_ARG, "spherical handle required");
  if (!phi || !out) return fail(PS_ERR_INVALID_ARG, "NULL buffer");
  cudaStream_t st = (cudaStream_t)stream;
  TRY(launch_sph_apply(h->sd, h->stab, phi, out, st));
  TRY(cudaStreamSynchronize(st));
  return PS_OK;
}

}  // extern "C"
