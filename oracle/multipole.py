"""Multipole open boundary (oracle), Sec. 2.2.

Eq. outer_multipole:  q_lm = sum_cells dV sqrt(4 pi/(2l+1)) rho(x') r'^l Y_lm(x')
Eq. outer_expansion:  Phi(x) = -G sum_{l<=lmax, |m|<=l} q_lm r^-(l+1)
                                  sqrt(4 pi/(2l+1)) Y_lm(x)

Y_lm are the real orthonormal spherical harmonics with the cosine functions
at m >= 0 and the sine functions at m < 0:
    m > 0:  sqrt(2) N_lm P_l^m(cos t) cos(m p)
    m = 0:  N_l0 P_l(cos t)
    m < 0:  sqrt(2) N_l|m| P_l^|m|(cos t) sin(|m| p)
    N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
P_l^m is the associated Legendre function without the Condon-Shortley phase
(the phase cancels in the product q_lm Y_lm).  Coefficients are stored at
index l*l + l + m.  Here this is evaluated directly per node in spherical
coordinates about the expansion origin.

Eq. inner_multipole / Eq. inner_expansion (spherical grids with r_in > 0):
    qbar_lm = sum_cells dV sqrt(4 pi/(2l+1)) rho(x') r'^-(l+1) Y_lm(x'),
    Phi(x) = -G sum qbar_lm r^l sqrt(4 pi/(2l+1)) Y_lm(x),
the expansion of the potential inside the innermost mass, written on the inner
ghost shell r_{-1} = 2 r_0 - r_1 when the inner boundary is this one instead of
the Neumann mirror.

Cartesian grids: the sum runs over interior nodes with dV = hx hy hz; the
potential is written on every non-interior node (the boundary layer and, for
the 13-point stencil, the ghost layer).  Spherical grids: dV = r^2 sin(theta)
dr dtheta dphi with midpoint spacings dr_i = (r_{i+1} - r_{i-1})/2, origin at
r = 0, potential written on the outer ghost shell.
"""
from __future__ import annotations

import math

import numpy as np

from .grid import CartGrid


def idx(l: int, m: int) -> int:
    return l * l + l + m


def assoc_legendre(lmax: int, x: np.ndarray):
    """P[l][m](x) for 0 <= m <= l <= lmax, no Condon-Shortley phase, from
    P_m^m = (2m-1)!! (1-x^2)^(m/2), P_{m+1}^m = (2m+1) x P_m^m,
    (l-m) P_l^m = (2l-1) x P_{l-1}^m - (l+m-1) P_{l-2}^m."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P = [[None] * (lmax + 1) for _ in range(lmax + 1)]
    pmm = np.ones_like(x)
    for m in range(lmax + 1):
        if m > 0:
            pmm = pmm * (2 * m - 1) * s
        P[m][m] = pmm
        if m + 1 <= lmax:
            P[m + 1][m] = (2 * m + 1) * x * pmm
        for l in range(m + 2, lmax + 1):
            P[l][m] = ((2 * l - 1) * x * P[l - 1][m] - (l + m - 1) * P[l - 2][m]) / (l - m)
    return P


def real_sph_harm(lmax: int, theta: np.ndarray, phi: np.ndarray):
    """List Y[l*l+l+m] of real orthonormal spherical harmonics."""
    P = assoc_legendre(lmax, np.cos(theta))
    Y = [None] * ((lmax + 1) ** 2)
    for l in range(lmax + 1):
        for m in range(0, l + 1):
            N = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            if m == 0:
                Y[idx(l, 0)] = N * P[l][0]
            else:
                Y[idx(l, m)] = math.sqrt(2.0) * N * P[l][m] * np.cos(m * phi)
                Y[idx(l, -m)] = math.sqrt(2.0) * N * P[l][m] * np.sin(m * phi)
    return Y


def _spherical(dx, dy, dz):
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    with np.errstate(invalid="ignore", divide="ignore"):
        ct = np.where(r > 0, dz / np.where(r > 0, r, 1.0), 1.0)
    theta = np.arccos(np.clip(ct, -1.0, 1.0))
    phi = np.arctan2(dy, dx)
    return r, theta, phi


def moments_points(values_dv: np.ndarray, dx, dy, dz, lmax: int) -> np.ndarray:
    """q_lm = sum_points (rho dV) sqrt(4pi/(2l+1)) r^l Y_lm."""
    r, theta, phi = _spherical(dx, dy, dz)
    Y = real_sph_harm(lmax, theta, phi)
    q = np.zeros((lmax + 1) ** 2)
    for l in range(lmax + 1):
        fac = math.sqrt(4 * math.pi / (2 * l + 1))
        rl = r ** l
        for m in range(-l, l + 1):
            q[idx(l, m)] = np.sum(values_dv * fac * rl * Y[idx(l, m)])
    return q


def potential_points(q: np.ndarray, dx, dy, dz, lmax: int, G: float) -> np.ndarray:
    """Eq. outer_expansion at points given relative to the origin."""
    r, theta, phi = _spherical(dx, dy, dz)
    Y = real_sph_harm(lmax, theta, phi)
    out = np.zeros_like(r)
    for l in range(lmax + 1):
        fac = math.sqrt(4 * math.pi / (2 * l + 1))
        rl = r ** (-(l + 1))
        for m in range(-l, l + 1):
            out += q[idx(l, m)] * rl * fac * Y[idx(l, m)]
    return -G * out


def _mesh(grid: CartGrid, origin):
    x = grid.coords(0) - origin[0]
    y = grid.coords(1) - origin[1]
    z = grid.coords(2) - origin[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def moments_cartesian(rho: np.ndarray, grid: CartGrid, origin, lmax: int) -> np.ndarray:
    X, Y, Z = _mesh(grid, origin)
    I = grid.interior
    dV = grid.h[0] * grid.h[1] * grid.h[2]
    return moments_points(rho[I] * dV, X[I], Y[I], Z[I], lmax)


def boundary_mask(grid: CartGrid) -> np.ndarray:
    m = np.ones(grid.shape, dtype=bool)
    m[grid.interior] = False
    return m


def apply_cartesian_bc(phi: np.ndarray, grid: CartGrid, q: np.ndarray, origin, lmax: int,
                       G: float) -> None:
    """Write Eq. outer_expansion on every non-interior node of phi."""
    X, Y, Z = _mesh(grid, origin)
    m = boundary_mask(grid)
    phi[m] = potential_points(q, X[m], Y[m], Z[m], lmax, G)


def direct_legendre_potential(rho: np.ndarray, grid: CartGrid, origin, lmax: int, G: float,
                              points) -> np.ndarray:
    """Independent form of the truncated expansion via the addition theorem:
    -G sum_cells rho dV sum_{l<=lmax} r'^l / r^(l+1) P_l(cos gamma)."""
    X, Y, Z = _mesh(grid, origin)
    I = grid.interior
    dV = grid.h[0] * grid.h[1] * grid.h[2]
    src = np.stack([X[I].ravel(), Y[I].ravel(), Z[I].ravel()], axis=1)
    w = rho[I].ravel() * dV
    rs = np.linalg.norm(src, axis=1)
    out = []
    for p in points:
        p = np.asarray(p, dtype=np.float64)
        rp = np.linalg.norm(p)
        with np.errstate(invalid="ignore", divide="ignore"):
            cg = np.where(rs > 0, src @ p / (np.where(rs > 0, rs, 1.0) * rp), 1.0)
        coeffs = np.zeros(lmax + 1)
        total = 0.0
        for l in range(lmax + 1):
            coeffs[:] = 0.0
            coeffs[l] = 1.0
            Pl = np.polynomial.legendre.legval(cg, coeffs)
            total += np.sum(w * rs ** l * Pl) / rp ** (l + 1)
        out.append(-G * total)
    return np.array(out)


# ---------------------------------------------------------------- spherical grids

def radial_extended(r: np.ndarray):
    """Radii with one ghost on each side: r_{-1} = 2 r_0 - r_1 (mirror of the
    inner Neumann boundary) and r_N = r_{N-1}^2 / r_{N-2} (geometric
    continuation, the next node of a logarithmic grid)."""
    return np.concatenate([[2.0 * r[0] - r[1]], r, [r[-1] * r[-1] / r[-2]]])


def moments_spherical(rho: np.ndarray, r, th, ph, lmax: int) -> np.ndarray:
    """Moments over all unknown nodes of the spherical grid (ghosted layout
    (Nphi+2, Ntheta+2, Nr+2), r fastest)."""
    re = radial_extended(r)
    dr = 0.5 * (re[2:] - re[:-2])
    dth = math.pi / th.size
    dph = 2.0 * math.pi / ph.size
    P, T, R = np.meshgrid(ph, th, r, indexing="ij")
    DR = np.broadcast_to(dr[None, None, :], R.shape)
    dV = R * R * np.sin(T) * DR * dth * dph
    vals = rho[1:-1, 1:-1, 1:-1] * dV
    dx = R * np.sin(T) * np.cos(P)
    dy = R * np.sin(T) * np.sin(P)
    dz = R * np.cos(T)
    return moments_points(vals, dx, dy, dz, lmax)


def spherical_outer_ghost(q: np.ndarray, r, th, ph, lmax: int, G: float) -> np.ndarray:
    """Potential on the outer ghost shell r_N, shape (Nphi, Ntheta)."""
    rN = radial_extended(r)[-1]
    P, T = np.meshgrid(ph, th, indexing="ij")
    dx = rN * np.sin(T) * np.cos(P)
    dy = rN * np.sin(T) * np.sin(P)
    dz = rN * np.cos(T)
    return potential_points(q, dx, dy, dz, lmax, G)


# ---------------------------------------------------------------- inner expansion (spherical)

def inner_moments_points(values_dv: np.ndarray, dx, dy, dz, lmax: int) -> np.ndarray:
    """Eq. inner_multipole: qbar_lm = sum (rho dV) sqrt(4pi/(2l+1)) r^-(l+1) Y_lm."""
    r, theta, phi = _spherical(dx, dy, dz)
    Y = real_sph_harm(lmax, theta, phi)
    q = np.zeros((lmax + 1) ** 2)
    for l in range(lmax + 1):
        fac = math.sqrt(4 * math.pi / (2 * l + 1))
        rl = r ** (-(l + 1))
        for m in range(-l, l + 1):
            q[idx(l, m)] = np.sum(values_dv * fac * rl * Y[idx(l, m)])
    return q


def inner_potential_points(qbar: np.ndarray, dx, dy, dz, lmax: int, G: float) -> np.ndarray:
    """Eq. inner_expansion at points given relative to the origin."""
    r, theta, phi = _spherical(dx, dy, dz)
    Y = real_sph_harm(lmax, theta, phi)
    out = np.zeros_like(r)
    for l in range(lmax + 1):
        fac = math.sqrt(4 * math.pi / (2 * l + 1))
        rl = r ** l
        for m in range(-l, l + 1):
            out += qbar[idx(l, m)] * rl * fac * Y[idx(l, m)]
    return -G * out


def _spherical_cells(rho, r, th, ph):
    re = radial_extended(r)
    dr = 0.5 * (re[2:] - re[:-2])
    dth = math.pi / th.size
    dph = 2.0 * math.pi / ph.size
    P, T, R = np.meshgrid(ph, th, r, indexing="ij")
    dV = R * R * np.sin(T) * np.broadcast_to(dr[None, None, :], R.shape) * dth * dph
    return (rho[1:-1, 1:-1, 1:-1] * dV, R * np.sin(T) * np.cos(P), R * np.sin(T) * np.sin(P),
            R * np.cos(T))


def inner_moments_spherical(rho: np.ndarray, r, th, ph, lmax: int) -> np.ndarray:
    vals, dx, dy, dz = _spherical_cells(rho, r, th, ph)
    return inner_moments_points(vals, dx, dy, dz, lmax)


def spherical_inner_ghost(qbar: np.ndarray, r, th, ph, lmax: int, G: float) -> np.ndarray:
    """Potential on the inner ghost shell r_{-1}, shape (Nphi, Ntheta)."""
    r0 = radial_extended(r)[0]
    P, T = np.meshgrid(ph, th, indexing="ij")
    return inner_potential_points(qbar, r0 * np.sin(T) * np.cos(P), r0 * np.sin(T) * np.sin(P),
                                  r0 * np.cos(T), lmax, G)


def direct_legendre_inner(vals, src, lmax: int, G: float, points) -> np.ndarray:
    """Independent form of the truncated inner expansion via the addition
    theorem: -G sum rho dV sum_{l<=lmax} r^l / r'^(l+1) P_l(cos gamma)."""
    rs = np.linalg.norm(src, axis=1)
    out = []
    for p in points:
        p = np.asarray(p, dtype=np.float64)
        rp = np.linalg.norm(p)
        cg = src @ p / (rs * rp)
        total = 0.0
        for l in range(lmax + 1):
            c = np.zeros(l + 1)
            c[l] = 1.0
            total += np.sum(vals * rp ** l / rs ** (l + 1) * np.polynomial.legendre.legval(cg, c))
        out.append(-G * total)
    return np.array(out)

