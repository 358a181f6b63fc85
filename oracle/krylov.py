"""Krylov solvers (oracle), Sec. 2.1.2.

Both work on flat float64 vectors of unknowns; the operator is a callback.

CG (A symmetric positive definite): x_m in x_0 + K_m(A, r_0) with the residual
orthogonal to K_m; inner products and operator applications only, with the
usual short recurrences:
    r = b - A x, p = r
    repeat: q = A p; alpha = (r.r)/(p.q); x += alpha p; r -= alpha q;
            stop when ||r|| <= tol * ref; beta = (r.r)_new/(r.r)_old;
            p = r + beta p.

BiCGSTAB (van der Vorst; non-symmetric A, here the spherical Laplacian) with
right preconditioning by B^-1 = diag(A)^-1 (the preconditioner is applied to a
vector, never formed as a product, Sec. 2.1.2):
    r = b - A x, rhat = r, p = r, rho = rhat.r
    repeat: phat = B^-1 p; v = A phat; alpha = rho / (rhat.v);
            s = r - alpha v; if ||s|| <= tol*ref: x += alpha phat, stop;
            shat = B^-1 s; t = A shat; omega = (t.s)/(t.t);
            x += alpha phat + omega shat; r = s - omega t;
            stop when ||r|| <= tol*ref;
            rho_new = rhat.r; beta = (rho_new/rho)(alpha/omega);
            p = r + beta (p - omega v).
Iterations are counted as full passes of the loop body (a pass that stops at
the s check counts as one).

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


def bicgstab(apply_A, inv_diag: np.ndarray, b: np.ndarray, x0: np.ndarray, tol: float,
             max_iter: int, ref: float, dot=numpy_dot) -> KrylovResult:
    x = x0.copy()
    r = b - apply_A(x)
    hist = [math.sqrt(dot(r, r)) / ref]
    if hist[-1] <= tol:
        return KrylovResult(x, 0, True, hist)
    rhat = r.copy()
    p = r.copy()
    rho = dot(rhat, r)
    for it in range(1, max_iter + 1):
        phat = inv_diag * p
        v = apply_A(phat)
        alpha = rho / dot(rhat, v)
        s = r - alpha * v
        snorm = math.sqrt(dot(s, s)) / ref
        if snorm <= tol:
            x += alpha * phat
            hist.append(snorm)
            return KrylovResult(x, it, True, hist)
        shat = inv_diag * s
        t = apply_A(shat)
        omega = dot(t, s) / dot(t, t)
        x += alpha * phat + omega * shat
        r = s - omega * t
        hist.append(math.sqrt(dot(r, r)) / ref)
        if hist[-1] <= tol:
            return KrylovResult(x, it, True, hist)
        rho_new = dot(rhat, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        rho = rho_new
    return KrylovResult(x, max_iter, False, hist)
