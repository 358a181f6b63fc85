"""Krylov solvers (oracle), Sec. 2.1.2.

Both work on flat float64 vectors of unknowns; the operator is a callback.

CG (A symmetric positive definite): x_m in x_0 + K_m(A, r_0) with the residual
orthogonal to K_m; inner products and operator applications only, with the
usual short recurrences:
    r = b - A x, p = r
    repeat: q = A p; alpha = (r.r)/(p.q); x += alpha p; r -= alpha q;
            stop when ||r|| <= tol * ref; beta = (r.r)_new/(r.r)_old;
            p = r + beta p.

Preconditioned CG with the multicolour Gauss-Seidel preconditioner of
Sec. 2.1.2 (see multigrid.pcg_on_grid for B): the same recurrences with
z = B^-1 r in place of r in the direction and in rho = r.z.

BiCGSTAB (van der Vorst; non-symmetric A, here the spherical Laplacian) with
right preconditioning by B^-1 = diag(A)^-1 (the preconditioner is applied to a
vector, never formed as a product, Sec. 2.1.2):
    r = b - A x, rhat = r, p = r, rho = rhat.r
    repeat: phat = B^-1 p; v = A phat; alpha = rho / (rhat.v);
            s = r - alpha v; shat = B^-1 s; t = A shat; omega = (t.s)/(t.t);
            x += alpha phat + omega shat; r = s - omega t;
            rho_new = rhat.r; beta = (rho_new/rho)(alpha/omega);
            p = r + beta (p - omega v).
Iterations are counted as passes of the loop body.
Stopping on the true residual (Sleijpen and van der Vorst's residual
replacement, "reliable updating"): the recursively updated r drifts away from
b - A x on graded spherical grids (at 64x32x64 with r_in = 0.01 the recursion
reports 8e-11 while b - A x is 6e-10), so whenever ||r|| has dropped to
`replace` times its largest value since the last replacement, claims the
tolerance, or the iteration budget ends, r is replaced by b - A x, and every
stopping decision is taken on such a replaced residual.  The iterate is
updated group-wise (their companion remedy): the increments
alpha phat + omega shat accumulate in z, which is added to x only at a
replacement, so x is rounded once per replacement instead of once per
iteration (on the spherical grid the pole coefficients amplify every rounding
of x by up to 1e11).  There is no separate exit at s: a pass always completes.
Breakdowns: a non-finite alpha is taken as 0 (s = r), a zero or non-finite
omega as 0 (r = s); after either, or when rhat.r is exactly 0, the shadow
residual and the search direction restart from the current residual
(rhat = p = r, rho = r.r).

`dot` selects how inner products are summed: numpy's (default) or exactly
rounded (math.fsum).  BiCGSTAB's iteration count on graded spherical grids
depends on such rounding choices, so tests use both to measure the spread a
correct implementation may show.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class KrylovResult:
    x: np.ndarray
    iterations: int
    converged: bool
    history: list = field(default_factory=list)   # relative residual per iteration


def numpy_dot(a, b):
    return float(a @ b)


def exact_dot(a, b):
    return math.fsum(a * b)


def cg(apply_A, b: np.ndarray, x0: np.ndarray, tol: float, max_iter: int,
       ref: float, dot=numpy_dot) -> KrylovResult:
    x = x0.copy()
    r = b - apply_A(x)
    rr = dot(r, r)
    hist = [np.sqrt(rr) / ref]
    if hist[-1] <= tol:
        return KrylovResult(x, 0, True, hist)
    p = r.copy()
    for it in range(1, max_iter + 1):
        q = apply_A(p)
        alpha = rr / dot(p, q)
        x += alpha * p
        r -= alpha * q
        rr_new = dot(r, r)
        hist.append(np.sqrt(rr_new) / ref)
        if hist[-1] <= tol:
            return KrylovResult(x, it, True, hist)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    return KrylovResult(x, max_iter, False, hist)


def pcg(apply_A, apply_Minv, b: np.ndarray, x0: np.ndarray, tol: float, max_iter: int,
        ref: float, dot=numpy_dot) -> KrylovResult:
    """Preconditioned CG (Sec. 2.1.2: the iteration for A B^-1, B^-1 applied to a
    vector): z = B^-1 r, p = z, rho = r.z; q = A p, alpha = rho/(p.q),
    x += alpha p, r -= alpha q; stop on ||r|| <= tol * ref (the unpreconditioned
    residual, as for CG); z = B^-1 r, beta = (r.z)_new / rho, p = z + beta p."""
    x = x0.copy()
    r = b - apply_A(x)
    rr = dot(r, r)
    hist = [np.sqrt(rr) / ref]
    if hist[-1] <= tol:
        return KrylovResult(x, 0, True, hist)
    z = apply_Minv(r)
    p = z.copy()
    rho = dot(r, z)
    for it in range(1, max_iter + 1):
        q = apply_A(p)
        alpha = rho / dot(p, q)
        x += alpha * p
        r -= alpha * q
        hist.append(np.sqrt(dot(r, r)) / ref)
        if hist[-1] <= tol:
            return KrylovResult(x, it, True, hist)
        z = apply_Minv(r)
        rho_new = dot(r, z)
        beta = rho_new / rho
        rho = rho_new
        p = z + beta * p
    return KrylovResult(x, max_iter, False, hist)


def _div(a: float, b: float) -> float:
    """IEEE quotient (inf / nan instead of an exception)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return float(np.float64(a) / np.float64(b))


def bicgstab(apply_A, inv_diag: np.ndarray, b: np.ndarray, x0: np.ndarray, tol: float,
             max_iter: int, ref: float, dot=numpy_dot, replace: float = 0.01,
             restart: bool = True) -> KrylovResult:
    """restart=False drops the breakdown rules (for tests).  history holds the
    relative residual after every pass (the true one after a replacement)."""
    x = x0.copy()
    r = b - apply_A(x)
    rr = dot(r, r)
    hist = [math.sqrt(rr) / ref]
    if hist[-1] <= tol:
        return KrylovResult(x, 0, True, hist)
    rhat = r.copy()
    p = r.copy()
    rho = dot(rhat, r)
    rmax = math.sqrt(rr)
    z = np.zeros_like(x)
    for it in range(1, max_iter + 1):
        phat = inv_diag * p
        v = apply_A(phat)
        alpha = _div(rho, dot(rhat, v))
        broke = restart and not math.isfinite(alpha)
        if broke:
            alpha = 0.0
        s = r - alpha * v
        shat = inv_diag * s
        t = apply_A(shat)
        omega = _div(dot(t, s), dot(t, t))
        if restart and not (math.isfinite(omega) and omega != 0.0):
            broke = True
            omega = 0.0
        z += alpha * phat + omega * shat
        r = s - omega * t
        rr = dot(r, r)
        rn = math.sqrt(rr)
        if (not math.isfinite(rn) or broke or rn <= replace * rmax or rn / ref <= tol
                or it == max_iter):
            x += z
            z[:] = 0.0
            r = b - apply_A(x)
            rr = dot(r, r)
            rn = math.sqrt(rr)
            rmax = rn
            hist.append(rn / ref)
            if rn / ref <= tol:
                return KrylovResult(x, it, True, hist)
            if not math.isfinite(rn):
                return KrylovResult(x, it, False, hist)
        else:
            rmax = max(rmax, rn)
            hist.append(rn / ref)
        rho_new = dot(rhat, r)
        if restart and (broke or rho_new == 0.0):
            rhat = r.copy()
            p = r.copy()
            rho = rr
            continue
        beta = _div(rho_new, rho) * _div(alpha, omega)
        p = r + beta * (p - omega * v)
        rho = rho_new
    return KrylovResult(x, max_iter, False, hist)
