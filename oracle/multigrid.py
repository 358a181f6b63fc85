"""Geometric multigrid V-cycle and FP64 iterative refinement (oracle).

Sec. 2.1.3 writes the V-cycle error operator recursively:
    E_i = S^nu1 (I - P E_{i+1} R A_i) S^nu2,   E_N = A_N^-1,
i.e. pre-smooth nu1 times, restrict the residual, solve the coarse error
equation (recursively; the coarsest one by CG), prolong and add the
correction, post-smooth nu2 times.  The coarse operators here are the same
stencil rediscretised with h_c = 2h (geometric MG); the coarsest level is
solved by CG to relative residual `coarse_tol` (or at most one iteration per
coarse unknown).  Sec. 2.1.3 notes that solving the coarse problem to a
relative accuracy of about the convergence factor rho keeps the asymptotic
rate and that reducing it much further is wasted work; the V(2,2) cycles here
have rho ~ 0.075, and coarse_tol = 1e-2 stays an order of magnitude below it.
The smoother is the multicolour Gauss-Seidel sweep with colours in ascending
order in both legs.

Eq. rho: the mean convergence factor after m cycles is
(||r_m|| / ||r_0||)^(1/m).

Iterative refinement (the mixed-precision scheme restated in float64): the
outer loop forms r = f - A phi, solves A e = r approximately by `inner` V-cycles
from e = 0 with zero boundary data, and adds e to phi.  In exact arithmetic one
inner V-cycle per outer step reproduces the plain MG iteration.
"""
from __future__ import annotations

import numpy as np

from . import krylov
from .grid import CartGrid, hierarchy
from .operators import laplacian, norm2, reference_norm, residual
from .smoothers import sweep
from .transfer import prolong, restrict

COARSE_TOL = 1e-2


def cg_on_grid(phi: np.ndarray, f: np.ndarray, grid: CartGrid, tol: float, max_iter: int):
    """CG for A phi = f on one grid, boundary data of phi held fixed.

    A is negative definite, so CG runs on the SPD system -A_0 x = -(f - A b)
    where A_0 is the operator with zero boundary data and b the boundary part.
    """
    I = grid.interior
    shape_int = phi[I].shape

    def apply_spd(v):
        full = grid.zeros()
        full[I] = v.reshape(shape_int)
        return -laplacian(full, grid)[I].ravel()

    bpart = phi.copy()
    bpart[I] = 0.0
    rhs = -(f[I] - laplacian(bpart, grid)[I]).ravel()
    ref = reference_norm(phi, f, grid)
    if ref == 0.0:
        ref = 1.0
    res = krylov.cg(apply_spd, rhs, phi[I].ravel().copy(), tol, max_iter, ref)
    phi[I] = res.x.reshape(shape_int)
    return res


def sgs_preconditioner(grid: CartGrid):
    """B^-1 of Sec. 2.1.2's multicolour Gauss-Seidel preconditioner for the SPD
    matrix -A_0 (zero boundary), as a function of a flat residual vector.

    The paper writes B as the block lower triangular part of A in colour order
    (D + L) and solves with it block-wise, one colour at a time.  CG needs a
    symmetric positive definite B, so the reading taken here is the symmetric
    form B = (D + L) D^-1 (D + U): Gauss-Seidel colour passes on -A_0 z = r
    from z = 0 in ascending colour order (that is (D + L)^-1 r), then in
    descending order; the first descending pass would repeat the last
    ascending one exactly (its operands are unchanged), so it is skipped:
    2 ncol - 1 passes."""
    from .smoothers import ncolours, sweep_colour
    ncol = ncolours(grid.order)
    I = grid.interior
    shape_int = grid.zeros()[I].shape

    def apply(r):
        z = grid.zeros()
        rhs = grid.zeros()
        rhs[I] = -r.reshape(shape_int)      # A_0 z = -r  <=>  -A_0 z = r
        for c in list(range(ncol)) + list(range(ncol - 2, -1, -1)):
            sweep_colour(z, rhs, grid, c, 1.0, ncol)
        return z[I].ravel().copy()
    return apply


def pcg_on_grid(phi: np.ndarray, f: np.ndarray, grid: CartGrid, tol: float, max_iter: int):
    """Multicolour-Gauss-Seidel-preconditioned CG for A phi = f (boundary data of
    phi fixed), on the SPD system -A_0 x = -(f - A b) as cg_on_grid."""
    I = grid.interior
    shape_int = phi[I].shape

    def apply_spd(v):
        full = grid.zeros()
        full[I] = v.reshape(shape_int)
        return -laplacian(full, grid)[I].ravel()

    bpart = phi.copy()
    bpart[I] = 0.0
    rhs = -(f[I] - laplacian(bpart, grid)[I]).ravel()
    ref = reference_norm(phi, f, grid)
    if ref == 0.0:
        ref = 1.0
    res = krylov.pcg(apply_spd, sgs_preconditioner(grid), rhs, phi[I].ravel().copy(), tol,
                     max_iter, ref)
    phi[I] = res.x.reshape(shape_int)
    return res


def vcycle(levels, l: int, phi: np.ndarray, f: np.ndarray, nu1: int, nu2: int,
           omega: float = 1.0, coarse_tol: float = COARSE_TOL) -> None:
    grid = levels[l]
    if l == len(levels) - 1:
        n_unknowns = int(np.prod([v - 1 for v in grid.n]))
        cg_on_grid(phi, f, grid, coarse_tol, n_unknowns)
        return
    for _ in range(nu1):
        sweep(phi, f, grid, omega)
    r = residual(phi, f, grid)
    coarse = levels[l + 1]
    fc = restrict(r, grid, coarse)
    ec = coarse.zeros()
    vcycle(levels, l + 1, ec, fc, nu1, nu2, omega, coarse_tol)
    phi += prolong(ec, coarse, grid)
    for _ in range(nu2):
        sweep(phi, f, grid, omega)


def mg_solve(phi: np.ndarray, f: np.ndarray, grid: CartGrid, tol: float, max_iter: int,
             nu1: int = 2, nu2: int = 2, omega: float = 1.0, coarse_tol: float = COARSE_TOL):
    """V(nu1,nu2) cycles until ||f - A phi|| <= tol * ref; returns
    (cycles, converged, history of relative residuals)."""
    levels = hierarchy(grid)
    ref = reference_norm(phi, f, grid)
    if ref == 0.0:
        ref = 1.0
    hist = [norm2(residual(phi, f, grid), grid) / ref]
    if hist[-1] <= tol:
        return 0, True, hist
    for it in range(1, max_iter + 1):
        vcycle(levels, 0, phi, f, nu1, nu2, omega, coarse_tol)
        hist.append(norm2(residual(phi, f, grid), grid) / ref)
        if hist[-1] <= tol:
            return it, True, hist
    return max_iter, False, hist


def ir_solve(phi: np.ndarray, f: np.ndarray, grid: CartGrid, tol: float, max_iter: int,
             nu1: int = 2, nu2: int = 2, inner: int = 1, coarse_tol: float = COARSE_TOL):
    """Iterative refinement around `inner` V-cycles on the error equation."""
    levels = hierarchy(grid)
    ref = reference_norm(phi, f, grid)
    if ref == 0.0:
        ref = 1.0
    hist = []
    for it in range(0, max_iter + 1):
        r = residual(phi, f, grid)
        hist.append(norm2(r, grid) / ref)
        if hist[-1] <= tol:
            return it, True, hist
        if it == max_iter:
            break
        e = grid.zeros()
        for _ in range(inner):
            vcycle(levels, 0, e, r, nu1, nu2, 1.0, coarse_tol)
        phi[grid.interior] += e[grid.interior]
    return max_iter, False, hist


def convergence_factor(hist) -> float:
    """Eq. rho over the recorded history (m = number of cycles)."""
    m = len(hist) - 1
    if m <= 0 or hist[0] == 0.0:
        return 0.0
    return float((hist[-1] / hist[0]) ** (1.0 / m))
