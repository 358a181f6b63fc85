"""GB300-native iterative Poisson solvers for self-gravity (arXiv 2605.03563).

Python face of libpoisson.so: tensors (torch, on the current CUDA device)
are passed to the C ABI by pointer together with torch's current stream.
Nothing here computes; every step of every solve runs in the CUDA library.

    from paper_2605_03563_gb300 import CartesianSolver
    s = CartesianSolver(256, bc="multipole", lmax=4)
    info = s.solve(rho, phi, tol=1e-10, method="mg")
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

from . import capi
from .capi import lib, check

__all__ = ["CartesianSolver", "SphericalSolver", "SolveInfo", "ops", "capi", "workspace_bytes"]

METHODS = {"sor": capi.PS_SOR, "cg": capi.PS_CG, "pcg": capi.PS_PCG, "mg": capi.PS_MG, "bicgstab": capi.PS_BICGSTAB}
PRECISIONS = {"fp64": capi.PS_FP64, "mixed_fp32": capi.PS_MIXED_FP32, "mixed_bf16": capi.PS_MIXED_BF16}
# SOR weights: the given omega, Eq. omega_n's Chebyshev sequence, omega_opt of Eq. 3
SOR_SCHEDULES = {"fixed": 0, "chebyshev": 1, "optimal": 2}


@dataclass
class SolveInfo:
    status: int
    iterations: int
    rel_residual: float
    rho_conv: float
    t_mp_ms: float
    t_iter_ms: float
    inner_cycles: int
    coarse_iterations: int
    kernel_launches: int
    moments: list = field(default_factory=list)

    @property
    def converged(self) -> bool:
        return self.status == capi.PS_OK

    @staticmethod
    def from_c(info: capi.PsInfo, nmom: int) -> "SolveInfo":
        return SolveInfo(info.status, info.iterations, info.rel_residual, info.rho_conv,
                         info.t_mp_ms, info.t_iter_ms, info.inner_cycles, info.coarse_iterations,
                         info.kernel_launches, list(info.moments[:nmom]))


def _ptr(t, dtype_name="float64"):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if str(t.dtype).replace("torch.", "") != dtype_name:
        raise ValueError(f"tensor dtype must be {dtype_name}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def workspace_bytes(n, order=2, lmax=4, prec="fp64", lo=(0, 0, 0), hi=(1, 1, 1)) -> int:
    g = capi.make_grid(n, lo, hi)
    return int(lib().poisson_workspace_bytes(C.byref(g), order, lmax, PRECISIONS[prec]))


class _Handle:
    def __init__(self):
        self._h = C.c_void_p()

    def close(self):
        if self._h:
            lib().poisson_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, enable=True):
        """Record CUDA-event timings of the hot kernels of this handle's solves."""
        check(lib().poisson_profile_enable(self._h, 1 if enable else 0), "poisson_profile_enable")

    def profile_read(self):
        """Per-kernel {launches, total_ms, avg_ms, bytes_per_launch, ops_per_launch, fp64}."""
        buf = (capi.PsKernelStat * 32)()
        k = lib().poisson_profile_read(self._h, buf, 32)
        if k < 0:
            raise capi.PoissonError(capi.PS_ERR_CUDA, "poisson_profile_read")
        out = {}
        for i in range(min(k, 32)):
            e = buf[i]
            out[e.name.decode()] = dict(launches=e.launches, total_ms=e.total_ms,
                                        avg_ms=e.total_ms / max(e.launches, 1),
                                        bytes_per_launch=e.bytes_per_launch,
                                        ops_per_launch=e.ops_per_launch, fp64=bool(e.fp64),
                                        variant=e.variant)
        return out

    # ---- tuned settings (poisson_set_tuning)
    def set_tuning(self, prec, nu1=2, nu2=2, inner_cycles=1, tile_min_n=0, sweep_tile=0, restrict_tile=0):
        """Install the tuned multigrid settings used by solves with tuned=True."""
        t = capi.PsTuning(int(nu1), int(nu2), int(inner_cycles), int(tile_min_n), int(sweep_tile),
                          int(restrict_tile))
        check(lib().poisson_set_tuning(self._h, PRECISIONS[prec], C.byref(t)), "poisson_set_tuning")

    def clear_tuning(self, prec):
        check(lib().poisson_set_tuning(self._h, PRECISIONS[prec], None), "poisson_set_tuning")

    def get_tuning(self, prec):
        """The installed tuning of a precision as a dict, or None."""
        t = capi.PsTuning()
        is_set = C.c_int()
        check(lib().poisson_get_tuning(self._h, PRECISIONS[prec], C.byref(t), C.byref(is_set)),
              "poisson_get_tuning")
        if not is_set.value:
            return None
        return dict(nu1=t.nu1, nu2=t.nu2, inner_cycles=t.inner_cycles, tile_min_n=t.tile_min_n,
                    sweep_tile=t.sweep_tile, restrict_tile=t.restrict_tile)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- asynchronous, steppable solves (continuous batching)
    def begin(self, rho, phi, tol=1e-10, method="mg", prec="fp64", omega=1.0, nu1=2, nu2=2,
              max_iter=100, inner_cycles=1, stream=None, tile_min_n=0, sor_schedule="fixed",
              compact_order=0, tuned=False):
        """Start a solve whose state stays on the device; rho/phi must stay alive until end()."""
        self._opts = capi.PsSolveOpts(METHODS[method], PRECISIONS[prec], float(omega), int(nu1),
                                      int(nu2), int(max_iter), int(inner_cycles), _stream(stream),
                                      int(tile_min_n), SOR_SCHEDULES[sor_schedule], int(compact_order),
                                      1 if tuned else 0)
        self._keep = (rho, phi)
        check(lib().poisson_solve_begin(self._h, _ptr(rho), _ptr(phi), float(tol),
                                        C.byref(self._opts)), "poisson_solve_begin")

    def step(self, max_iterations=1):
        """Enqueue up to max_iterations more iterations (no host synchronisation)."""
        check(lib().poisson_solve_step(self._h, int(max_iterations)), "poisson_solve_step")

    def poll(self):
        """Wait for this solve's stream; returns (done, SolveInfo so far)."""
        done = C.c_int()
        info = capi.PsInfo()
        check(lib().poisson_solve_poll(self._h, C.byref(done), C.byref(info)), "poisson_solve_poll")
        return bool(done.value), SolveInfo.from_c(info, 0)

    def end(self):
        """Copy the iterate back to phi and return the final SolveInfo."""
        info = capi.PsInfo()
        st = lib().poisson_solve_end(self._h, C.byref(info))
        check(st, "poisson_solve_end", allow=(capi.PS_OK, capi.PS_NOT_CONVERGED, capi.PS_DIVERGED))
        self._keep = None
        nmom = (self.lmax + 1) ** 2 if getattr(self, "multipole", False) else 0
        return SolveInfo.from_c(info, min(nmom, 81))

    def _solve(self, rho, phi, tol, method, prec, omega, nu1, nu2, max_iter, inner_cycles,
               stream, nmom, tile_min_n=0, sor_schedule="fixed", compact_order=0, tuned=False):
        opts = capi.PsSolveOpts(METHODS[method], PRECISIONS[prec], float(omega), int(nu1),
                                int(nu2), int(max_iter), int(inner_cycles), _stream(stream),
                                int(tile_min_n), SOR_SCHEDULES[sor_schedule], int(compact_order),
                                1 if tuned else 0)
        info = capi.PsInfo()
        st = lib().poisson_solve(self._h, _ptr(rho), _ptr(phi), float(tol), C.byref(opts),
                                 C.byref(info))
        check(st, "poisson_solve", allow=(capi.PS_OK, capi.PS_NOT_CONVERGED, capi.PS_DIVERGED))
        return SolveInfo.from_c(info, nmom)


class CartesianSolver(_Handle):
    """Uniform Cartesian grid with n intervals per axis on [lo, hi]^3.

    Fields are float64 tensors of shape (nz+2g-1, ny+2g-1, nx+2g-1), g = order/2.
    bc = "dirichlet" (phi carries the boundary data) or "multipole" (Sec. 2.2)."""

    def __init__(self, n, order=2, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc="dirichlet",
                 lmax=4, origin=None, G=1.0):
        super().__init__()
        self.n = (n, n, n) if isinstance(n, int) else tuple(n)
        self.order, self.lmax = order, lmax
        if origin is None:
            origin = tuple(0.5 * (lo[a] + hi[a]) for a in range(3))
        grid = capi.make_grid(self.n, lo, hi)
        b = capi.PsBC(capi.PS_BC_MULTIPOLE if bc == "multipole" else capi.PS_BC_DIRICHLET_GIVEN,
                      capi.PS_INNER_NONE, (C.c_double * 3)(*origin), float(G))
        self.multipole = bc == "multipole"
        check(lib().poisson_create(C.byref(grid), None, order, C.byref(b), lmax, C.byref(self._h)),
              "poisson_create")

    @property
    def shape(self):
        g = self.order // 2
        nx, ny, nz = self.n
        return (nz + 2 * g - 1, ny + 2 * g - 1, nx + 2 * g - 1)

    def solve(self, rho, phi, tol=1e-10, method="mg", prec="fp64", omega=1.0, nu1=2, nu2=2,
              max_iter=100, inner_cycles=1, stream=None, tile_min_n=0,
              sor_schedule="fixed", compact_order=0, tuned=False) -> SolveInfo:
        """tile_min_n: levels with at least this many intervals per axis use the TMA tile
        kernels (0 = library default, negative = never); results are bitwise identical.
        sor_schedule (method "sor"): "fixed" (omega), "chebyshev" (Eq. omega_n) or
        "optimal" (Eq. 3), the last two with rJ of Eq. 4.
        compact_order (method "mg", order-2 handle, equal spacings): 2, 4 or 6 selects the
        compact discretisation of that order with SPAI smoothing and Galerkin coarse
        operators (Sec. 2.1.3); 0 the 7-point / 13-point stencil with Gauss-Seidel.
        tuned (method "mg"): take nu1, nu2, inner_cycles, tile_min_n and the fused sweep's
        tile shape from the handle's tuning for prec (set_tuning, or use_table) when one
        is installed."""
        nmom = (self.lmax + 1) ** 2 if self.multipole else 0
        return self._solve(rho, phi, tol, method, prec, omega, nu1, nu2, max_iter, inner_cycles,
                           stream, min(nmom, 81), tile_min_n, sor_schedule, compact_order, tuned)

    def use_table(self, prec="fp64", tol=1e-10, table=None):
        """Install the autotuner's entry for this grid (n, order, prec, tol) from a table
        (dict or path; default: the package's table file) on the handle.  Returns the
        installed settings, or None when the table has no entry (the handle keeps the
        library defaults)."""
        from . import autotune
        if table is None or isinstance(table, str):
            table = autotune.load(table) if table else autotune.load()
        if len(set(self.n)) != 1:
            return None
        e = autotune.lookup(table, self.n[0], self.order, prec, tol)
        if not e:
            self.clear_tuning(prec)
            return None
        self.set_tuning(prec, e["nu1"], e["nu2"], e["inner"], e.get("tile_min_n", 0), e.get("sweep_tile", 0),
                        e.get("restrict_tile", 0))
        return self.get_tuning(prec)


class SphericalSolver(_Handle):
    """Spherical grid with node coordinates r (increasing), theta_j = (j+1/2) pi/Nt,
    phi_k = 2 pi k/Np; Neumann or multipole inner boundary, multipole or given outer boundary.
    Fields are float64 tensors of shape (Np+2, Nt+2, Nr+2) (r fastest)."""

    def __init__(self, r, theta, phi, bc="multipole", lmax=6, G=1.0, inner="neumann"):
        """inner: "neumann" (mirror ghost) or "multipole" (Dirichlet ghost from the inner
        expansion of Sec. 2.2)."""
        super().__init__()
        import numpy as np
        self._coords = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (r, theta, phi)]
        self.n = tuple(a.size for a in self._coords)
        self.lmax = lmax
        grid = capi.make_grid(self.n, kind=capi.PS_GRID_SPHERICAL)
        ptrs = (C.c_void_p * 3)(*[a.ctypes.data for a in self._coords])
        b = capi.PsBC(capi.PS_BC_MULTIPOLE if bc == "multipole" else capi.PS_BC_DIRICHLET_GIVEN,
                      capi.PS_INNER_MULTIPOLE if inner == "multipole" else capi.PS_INNER_NEUMANN,
                      (C.c_double * 3)(0, 0, 0), float(G))
        self.multipole = bc == "multipole"
        check(lib().poisson_create(C.byref(grid), C.cast(ptrs, C.POINTER(C.c_void_p)), 2,
                                   C.byref(b), lmax, C.byref(self._h)), "poisson_create")

    @property
    def shape(self):
        nr, nt, np_ = self.n
        return (np_ + 2, nt + 2, nr + 2)

    def solve(self, rho, phi, tol=1e-10, prec="fp64", max_iter=20000, inner_cycles=0,
              stream=None, method="bicgstab", omega=1.0, sor_schedule="chebyshev") -> SolveInfo:
        """method "bicgstab" (right-Jacobi BiCGSTAB) or "sor" (red-black SOR, FP64, with
        sor_schedule "fixed" (omega), "chebyshev" (Eq. omega_n) or "optimal" (Eq. 3), the
        last two per node with the local rJ of Eq. local_rjac)."""
        nmom = (self.lmax + 1) ** 2 if self.multipole else 0
        return self._solve(rho, phi, tol, method, prec, omega, 0, 0, max_iter, inner_cycles,
                           stream, min(nmom, 81), 0, sor_schedule)

    def apply(self, phi, out, stream=None):
        check(lib().ps_op_spherical_apply(self._h, _ptr(phi), _ptr(out), _stream(stream)),
              "ps_op_spherical_apply")


def solve_batch(solvers, rhos, phis, tols, method="mg", prec="fp64", nu1=2, nu2=2, max_iter=100,
                inner_cycles=1, stream=None, tile_min_n=0):
    """poisson_solve_batch over distinct CartesianSolver handles."""
    n = len(solvers)
    hs = (C.c_void_p * n)(*[s._h.value for s in solvers])
    rp = (C.c_void_p * n)(*[_ptr(r).value for r in rhos])
    pp = (C.c_void_p * n)(*[_ptr(p).value for p in phis])
    tl = (C.c_double * n)(*[float(t) for t in tols])
    opts = capi.PsSolveOpts(METHODS[method], PRECISIONS[prec], 1.0, nu1, nu2, max_iter,
                            inner_cycles, _stream(stream), int(tile_min_n))
    infos = (capi.PsInfo * n)()
    st = lib().poisson_solve_batch(hs, rp, pp, tl, n, C.byref(opts), infos)
    check(st, "poisson_solve_batch", allow=(capi.PS_OK, capi.PS_NOT_CONVERGED, capi.PS_DIVERGED))
    return [SolveInfo.from_c(infos[i], min(81, (s.lmax + 1) ** 2 if s.multipole else 0))
            for i, s in enumerate(solvers)]


class Batch:
    """Batched multigrid executor (poisson_batch_*): many CartesianSolver handles of
    different sizes advanced together by one CUDA-graph launch per step.

    add() starts a solve in a free slot and returns the slot; step(k) enqueues k
    V-cycles (FP64) or refinement steps (mixed_fp32) of every active solve; poll()
    returns per-slot (status, iterations) arrays (status -1 free, 0 running,
    1 converged, 2 budget exhausted, 3 diverged, 4 fault); remove(slot) copies the
    potential back and returns the SolveInfo."""

    def __init__(self, capacity, max_n, order=2, prec="fp64", nu1=2, nu2=2, inner_cycles=1):
        self._b = C.c_void_p()
        self.capacity = int(capacity)
        check(lib().poisson_batch_create(self.capacity, int(max_n), int(order), PRECISIONS[prec],
                                         int(nu1), int(nu2), int(inner_cycles), C.byref(self._b)),
              "poisson_batch_create")
        self._keep = {}

    def add(self, solver, rho, phi, tol=1e-10, max_iter=100) -> int:
        slot = C.c_int(-1)
        check(lib().poisson_batch_add(self._b, solver._h, _ptr(rho), _ptr(phi), float(tol),
                                      int(max_iter), C.byref(slot)), "poisson_batch_add")
        self._keep[slot.value] = (solver, rho, phi)
        return slot.value

    def step(self, iterations=1):
        check(lib().poisson_batch_step(self._b, int(iterations)), "poisson_batch_step")

    def poll(self):
        st = (C.c_int32 * self.capacity)()
        it = (C.c_int32 * self.capacity)()
        check(lib().poisson_batch_poll(self._b, st, it), "poisson_batch_poll")
        return list(st), list(it)

    def remove(self, slot) -> SolveInfo:
        info = capi.PsInfo()
        solver = self._keep[slot][0]
        st = lib().poisson_batch_remove(self._b, int(slot), C.byref(info))
        check(st, "poisson_batch_remove", allow=(capi.PS_OK, capi.PS_NOT_CONVERGED, capi.PS_DIVERGED))
        del self._keep[slot]
        nmom = (solver.lmax + 1) ** 2 if getattr(solver, "multipole", False) else 0
        return SolveInfo.from_c(info, min(nmom, 81))

    def close(self):
        if self._b:
            lib().poisson_batch_destroy(self._b)
            self._b = C.c_void_p()
            self._keep = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


from . import ops  # noqa: E402
