"""Compact stencils, SPAI smoothers and Galerkin coarse operators (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2.1.3: on isotropic Cartesian grids the Laplacian of order 2, 4 or 6 has
a compact discretisation of radius one; multigrid smooths it with the sparse
approximate inverse (SPAI) smoother of Eq. richardson,
    x <- (I - omega M A) x + omega M b,
M the radius-one symmetric stencil h^2 {alpha centre, beta faces, gamma edges,
delta corners} of Eq. Smoother with the coefficients of Table 1, and uses the
Galerkin coarse operators A_{i+1} = R A_i R^T.

Isotropic 27-point stencils are written by offset class: centre (0 nonzero
offsets), 6 faces (1), 12 edges (2), 8 corners (3).

Compact schemes L_h u = R_h f (f = 4 pi G rho, L_h ~ Laplacian), with weights
obtained by matching Taylor expansions on monomials (the paper cites Spotz's
compact schemes without printing them):
  order 2:  L = (-6, 1, 0, 0) / h^2,             R f = f;
  order 4:  L = (-24, 2, 1, 0) / (6 h^2),        R f = f/2 + (1/12) sum_faces f;
  order 6:  L = (-128, 14, 3, 1) / (30 h^2),     R f = f + h^2/12 lap f + h^4/360 lap^2 f
            + h^4/180 (f_xxyy + f_yyzz + f_zzxx), written on nodes as
            (67/120) f + (1/18) sum_faces f + (1/90) sum_edges f - (1/240) sum_{+-2 e_a} f
            (the +-2 offsets reach one layer past the node array at the first
            interior layer; that value is the cubic extrapolation
            4 f_0 - 6 f_1 + 4 f_2 - f_3 along the axis).
Readings (where the paper is silent): the SPAI step on L_h u = R_h f is
u <- u - omega M (R_h f - L_h u) (Eq. richardson for A = -L_h, which is SPD
as the positive M of Table 1 requires); the residual outside the unknowns is
zero; every level uses Table 1's coefficients with its own h; the Galerkin
operator is R A P with P = 8 R^T the prolongation in use (the paper's R A R^T
up to the constant c of P = c R^T; the coarse-grid correction needs R A P).
Table 1's row for order 6 prints delta equal to mu (0.0909), a garbled cell:
delta is taken as the value that minimises the LFA smoothing factor with the
printed omega, alpha, beta, gamma (DELTA6 below, which `lfa_mu` reproduces).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import krylov
from .grid import CartGrid, hierarchy
from .transfer import prolong, restrict

# L_h weights (times 1/h^2) and R_h weights by offset class
L_WEIGHTS = {2: (-6.0, 1.0, 0.0, 0.0),
             4: (-24.0 / 6.0, 2.0 / 6.0, 1.0 / 6.0, 0.0),
             6: (-128.0 / 30.0, 14.0 / 30.0, 3.0 / 30.0, 1.0 / 30.0)}
R_WEIGHTS = {2: (1.0, 0.0, 0.0, 0.0),
             4: (0.5, 1.0 / 12.0, 0.0, 0.0),
             6: (67.0 / 120.0, 1.0 / 18.0, 1.0 / 90.0, 0.0)}
R6_AXIS2 = -1.0 / 240.0

# Table 1: omega, alpha, beta, gamma, delta, mu
DELTA6 = 0.0151
TABLE1 = {2: (1.3699, 0.1432, 0.0284, 0.0081, 0.0025, 0.1888),
          4: (0.9363, 0.2807, 0.0329, 0.0166, 0.0044, 0.0828),
          6: (0.3543, 0.7064, 0.1005, 0.0363, DELTA6, 0.0909)}

OFFSETS = list(itertools.product((-1, 0, 1), repeat=3))


def offset_class(d) -> int:
    return sum(1 for v in d if v != 0)


def _view(a: np.ndarray, grid: CartGrid, d):
    """`a` at interior positions shifted by d = (dx, dy, dz)."""
    I = grid.interior
    sl = []
    for ax, s in zip((2, 1, 0), I):           # array axes z, y, x
        sl.append(slice(s.start + d[ax], s.stop + d[ax]))
    return a[tuple(sl)]


def apply27(u: np.ndarray, grid: CartGrid, w, scale: float = 1.0) -> np.ndarray:
    """scale * sum_d w[class(d)] u[p + d] on the interior (full-shape result)."""
    out = np.zeros_like(u)
    acc = np.zeros(u[grid.interior].shape)
    for d in OFFSETS:
        c = w[offset_class(d)]
        if c != 0.0:
            acc += c * _view(u, grid, d)
    out[grid.interior] = scale * acc
    return out


def check_isotropic(grid: CartGrid) -> float:
    h = grid.h
    if not (abs(h[0] - h[1]) <= 1e-14 * h[0] and abs(h[1] - h[2]) <= 1e-14 * h[0]):
        raise ValueError("compact stencils and SPAI smoothers need equal spacings")
    if grid.order != 2:
        raise ValueError("compact stencils use the radius-one layout (order 2 grid)")
    return h[0]


def compact_rhs(f: np.ndarray, grid: CartGrid, order: int) -> np.ndarray:
    """R_h f on the interior."""
    h = check_isotropic(grid)
    b = apply27(f, grid, R_WEIGHTS[order])
    if order == 6:
        # one extrapolated layer on every side for the +-2 offsets
        fe = np.pad(f, 1)
        for ax in range(3):
            lo = [slice(None)] * 3
            src = lambda k: tuple(slice(None) if a != ax else k for a in range(3))
            fe[src(0)] = (4 * fe[src(1)] - 6 * fe[src(2)] + 4 * fe[src(3)] - fe[src(4)])
            n = fe.shape[ax]
            fe[src(n - 1)] = (4 * fe[src(n - 2)] - 6 * fe[src(n - 3)] + 4 * fe[src(n - 4)] - fe[src(n - 5)])
        I = grid.interior
        acc = np.zeros(f[I].shape)
        for ax in range(3):
            for s in (-2, 2):
                sl = []
                for a, sI in zip((2, 1, 0), I):
                    off = s if a == ax else 0
                    sl.append(slice(sI.start + 1 + off, sI.stop + 1 + off))
                acc += fe[tuple(sl)]
        b[I] += R6_AXIS2 * acc
    return b


def galerkin(w_fine, h_fine: float):
    """Class weights of R A P on the coarse grid (as a stencil in absolute units,
    i.e. not divided by h^2), for a fine isotropic 27-point A = w / h_fine^2:
    built by prolonging a coarse delta, applying A and restricting; also returns
    the largest entry outside radius one (zero: the radius stays one)."""
    fine = CartGrid((8, 8, 8), (0.0, 0.0, 0.0), (8 * h_fine,) * 3, 2)
    coarse = fine.coarsen()
    ec = coarse.zeros()
    ec[2, 2, 2] = 1.0
    Pe = prolong(ec, coarse, fine)
    APe = apply27(Pe, fine, w_fine, 1.0 / h_fine ** 2)
    st = restrict(APe, fine, coarse)                  # column of R A P for coarse node (2,2,2)
    out = [[] for _ in range(4)]
    beyond = 0.0
    for kz in range(1, 4):
        for ky in range(1, 4):
            for kx in range(1, 4):
                d = (kx - 2, ky - 2, kz - 2)
                out[offset_class(d)].append(st[kz, ky, kx])
    for idx in itertools.product(range(coarse.shape[0]), repeat=3):
        if max(abs(v - 2) for v in idx) >= 2:
            beyond = max(beyond, abs(st[idx]))
    w = tuple(float(np.mean(v)) for v in out)
    spread = max(float(np.max(v) - np.min(v)) for v in out)
    return w, beyond, spread


def level_operators(levels, order: int):
    """Per level the class weights of A (absolute units) -- the compact stencil on
    the finest level, Galerkin products below."""
    h0 = levels[0].h[0]
    ops = [tuple(c / h0 ** 2 for c in L_WEIGHTS[order])]
    for l in range(1, len(levels)):
        hf = levels[l - 1].h[0]
        wf = tuple(c * hf ** 2 for c in ops[-1])           # back to "times 1/h^2" form
        w, _, _ = galerkin(wf, hf)
        ops.append(w)
    return ops


def spai_weights(order: int, h: float):
    om, a, b, g, d, _ = TABLE1[order]
    return om, (a * h * h, b * h * h, g * h * h, d * h * h)


def residual27(u, b, grid, wA):
    r = -apply27(u, grid, wA)
    r[grid.interior] += b[grid.interior]
    return r


def spai_step(u, b, grid, wA, order):
    """u <- u - omega M (b - A u) (Eq. richardson with A -> -L_h)."""
    om, wM = spai_weights(order, grid.h[0])
    r = residual27(u, b, grid, wA)
    u[grid.interior] -= om * apply27(r, grid, wM)[grid.interior]


def _coarse_cg(u, b, grid, wA, tol):
    I = grid.interior
    shp = u[I].shape

    def apply_spd(v):
        full = grid.zeros()
        full[I] = v.reshape(shp)
        return -apply27(full, grid, wA)[I].ravel()

    rhs = -b[I].ravel()
    ref = float(np.sqrt(rhs @ rhs)) or 1.0
    res = krylov.cg(apply_spd, rhs, u[I].ravel().copy(), tol, int(np.prod(shp)), ref)
    u[I] = res.x.reshape(shp)


def vcycle(levels, ops, l, u, b, nu1, nu2, order, coarse_tol):
    grid = levels[l]
    if l == len(levels) - 1:
        _coarse_cg(u, b, grid, ops[l], coarse_tol)
        return
    for _ in range(nu1):
        spai_step(u, b, grid, ops[l], order)
    r = residual27(u, b, grid, ops[l])
    coarse = levels[l + 1]
    bc = restrict(r, grid, coarse)
    ec = coarse.zeros()
    vcycle(levels, ops, l + 1, ec, bc, nu1, nu2, order, coarse_tol)
    u += prolong(ec, coarse, grid)
    for _ in range(nu2):
        spai_step(u, b, grid, ops[l], order)


def mg_solve(phi, f, grid: CartGrid, order: int, tol: float, max_iter: int, nu1: int = 3,
             nu2: int = 3, coarse_tol: float = 1e-2):
    """V(nu1,nu2) cycles with SPAI smoothing and Galerkin coarse operators for
    L_h phi = R_h f, boundary data of phi fixed; stop on
    ||R_h f - L_h phi|| <= tol ||R_h f - L_h phi0|| (phi0: boundary data only).
    Returns (cycles, converged, history)."""
    check_isotropic(grid)
    levels = hierarchy(grid)
    ops = level_operators(levels, order)
    b = compact_rhs(f, grid, order)
    I = grid.interior
    phi0 = phi.copy()
    phi0[I] = 0.0
    nrm = lambda u: float(np.sqrt(np.sum(residual27(u, b, grid, ops[0])[I] ** 2)))
    ref = nrm(phi0) or 1.0
    hist = [nrm(phi) / ref]
    if hist[-1] <= tol:
        return 0, True, hist
    for it in range(1, max_iter + 1):
        vcycle(levels, ops, 0, phi, b, nu1, nu2, order, coarse_tol)
        hist.append(nrm(phi) / ref)
        if hist[-1] <= tol:
            return it, True, hist
    return max_iter, False, hist


def lfa_mu(order: int, npts: int = 65, coeffs=None) -> float:
    """Smoothing factor max |1 - omega M~(k) A~(k)| over the high frequencies
    T = [-pi, pi]^3 minus [-pi/2, pi/2]^3, k sampled on an npts-point grid per
    axis that includes +-pi (A~ the symbol of -L_h h^2, M~ that of M / h^2)."""
    om, a, b, g, d, _ = TABLE1[order] if coeffs is None else coeffs
    k = np.linspace(-math.pi, math.pi, npts)
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    cx, cy, cz = np.cos(KX), np.cos(KY), np.cos(KZ)
    s1, s2, s3 = cx + cy + cz, cx * cy + cy * cz + cz * cx, cx * cy * cz
    w = L_WEIGHTS[order]
    A = -(w[0] + 2 * w[1] * s1 + 4 * w[2] * s2 + 8 * w[3] * s3)
    M = a + 2 * b * s1 + 4 * g * s2 + 8 * d * s3
    S = 1.0 - om * M * A
    hi = np.maximum(np.maximum(np.abs(KX), np.abs(KY)), np.abs(KZ)) > math.pi / 2 + 1e-12
    return float(np.max(np.abs(S[hi])))
