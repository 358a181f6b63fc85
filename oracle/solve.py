"""Whole-solve drivers (oracle) with the same inputs and outputs as the C ABI.

A solve takes the density rho and a potential field phi that carries the
initial guess on unknown nodes and Dirichlet data on boundary/ghost nodes.
The right-hand side of Eq. 1 / Eq. 2 is f = 4 pi G rho.  With the multipole
boundary (Sec. 2.2) the boundary values are first replaced by the truncated
outer expansion of the moments of rho.  Iterations stop when
||f - A phi||_2 <= tol * ||f - A phi0||_2, phi0 being phi with zero unknowns,
checked after every SOR step, CG/BiCGSTAB iteration or V-cycle; reaching
max_iter without that is "not converged" (Sec. 2.1: a warning, not an error).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import compact, multigrid, multipole
from .grid import CartGrid
from .operators import norm2, reference_norm, residual
from .smoothers import (ncolours, omega_first, omega_next, omega_opt, rjac_uniform, sweep,
                        sweep_colour)
from .spherical import SphericalOperator, bicgstab_solve, sor_solve_spherical


@dataclass
class SolveInfo:
    iterations: int
    converged: bool
    rel_residual: float
    rho_conv: float
    history: list = field(default_factory=list)
    moments: np.ndarray | None = None


def sor_solve(phi, f, grid: CartGrid, omega: float, tol: float, max_iter: int,
              schedule: str = "fixed"):
    """SOR steps (Sec. 2.1.1) until the relative residual reaches tol.
    schedule: "fixed" (the given omega), "opt" (Eq. 3 with rJ of Eq. 4) or
    "chebyshev" (omega_n of Eq. omega_n from n = 1, one n per colour pass)."""
    ref = reference_norm(phi, f, grid)
    if ref == 0.0:
        ref = 1.0
    hist = [norm2(residual(phi, f, grid), grid) / ref]
    if hist[-1] <= tol:
        return 0, True, hist
    ncol = ncolours(grid.order)
    rj = rjac_uniform(grid)
    w = omega_first(rj)
    for it in range(1, max_iter + 1):
        if schedule == "fixed":
            sweep(phi, f, grid, omega)
        elif schedule == "opt":
            sweep(phi, f, grid, omega_opt(rj))
        elif schedule == "chebyshev":
            for c in range(ncol):
                sweep_colour(phi, f, grid, c, w, ncol)
                w = omega_next(rj, w)
        else:
            raise ValueError(schedule)
        hist.append(norm2(residual(phi, f, grid), grid) / ref)
        if hist[-1] <= tol:
            return it, True, hist
    return max_iter, False, hist


def solve_cartesian(rho: np.ndarray, phi: np.ndarray, grid: CartGrid, method: str, tol: float,
                    max_iter: int = 10000, G: float = 1.0, bc: str = "dirichlet", lmax: int = 4,
                    origin=None, omega: float = 1.0, nu1: int = 2, nu2: int = 2,
                    inner: int = 1, sor_schedule: str = "fixed", compact_order: int = 0) -> SolveInfo:
    """method in {"sor", "cg", "pcg", "mg", "ir"}; phi is updated in place."""
    f = 4.0 * math.pi * G * rho
    q = None
    if bc == "multipole":
        if origin is None:
            origin = tuple(0.5 * (grid.lo[a] + grid.hi[a]) for a in range(3))
        q = multipole.moments_cartesian(rho, grid, origin, lmax)
        multipole.apply_cartesian_bc(phi, grid, q, origin, lmax, G)
    if method == "sor":
        it, conv, hist = sor_solve(phi, f, grid, omega, tol, max_iter, sor_schedule)
    elif method == "cg":
        res = multigrid.cg_on_grid(phi, f, grid, tol, max_iter)
        it, conv, hist = res.iterations, res.converged, res.history
    elif method == "pcg":
        res = multigrid.pcg_on_grid(phi, f, grid, tol, max_iter)
        it, conv, hist = res.iterations, res.converged, res.history
    elif method == "mg" and compact_order:
        # compact stencil of that order, SPAI smoothing, Galerkin coarse operators (Sec. 2.1.3)
        it, conv, hist = compact.mg_solve(phi, f, grid, compact_order, tol, max_iter, nu1, nu2)
    elif method == "mg":
        it, conv, hist = multigrid.mg_solve(phi, f, grid, tol, max_iter, nu1, nu2)
    elif method == "ir":
        it, conv, hist = multigrid.ir_solve(phi, f, grid, tol, max_iter, nu1, nu2, inner)
    else:
        raise ValueError(method)
    return SolveInfo(it, conv, hist[-1], multigrid.convergence_factor(hist), hist, q)


def solve_spherical(rho: np.ndarray, phi: np.ndarray, r, th, ph, tol: float,
                    max_iter: int = 20000, G: float = 1.0, bc: str = "multipole",
                    lmax: int = 6, exact_dots: bool = False, method: str = "bicgstab",
                    omega: float = 1.0, sor_schedule: str = "chebyshev",
                    inner_bc: str = "neumann", dot=None) -> SolveInfo:
    """Right-Jacobi BiCGSTAB (or red-black SOR) on the spherical grid; phi in
    the ghosted layout.  dot (BiCGSTAB): how inner products are summed, a
    callable (a, b) -> float; default numpy's, or exactly rounded with
    exact_dots."""
    op = SphericalOperator(r, th, ph, inner="dirichlet" if inner_bc == "multipole" else "neumann")
    f = 4.0 * math.pi * G * rho
    q = None
    if bc == "multipole":
        q = multipole.moments_spherical(rho, r, th, ph, lmax)
        phi[1:-1, 1:-1, -1] = multipole.spherical_outer_ghost(q, r, th, ph, lmax, G)
    if inner_bc == "multipole":
        qb = multipole.inner_moments_spherical(rho, r, th, ph, lmax)
        phi[1:-1, 1:-1, 0] = multipole.spherical_inner_ghost(qb, r, th, ph, lmax, G)
    if method == "sor":
        it, conv, hist = sor_solve_spherical(phi, f, op, tol, max_iter, sor_schedule, omega)
        return SolveInfo(it, conv, hist[-1], multigrid.convergence_factor(hist), hist, q)
    from . import krylov
    if dot is None:
        dot = krylov.exact_dot if exact_dots else krylov.numpy_dot
    res = bicgstab_solve(phi, f, op, tol, max_iter, dot=dot)
    return SolveInfo(res.iterations, res.converged, res.history[-1],
                     multigrid.convergence_factor(res.history), res.history, q)
