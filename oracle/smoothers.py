"""Multicolour Gauss-Seidel / SOR sweeps and the SOR weight (oracle).

Sec. 2.1.1: red-black Gauss-Seidel updates the two colours of a 3-D
checkerboard one after the other; SOR scales each Gauss-Seidel correction by
omega (0 < omega < 2; omega = 1 is Gauss-Seidel).  One SOR "step" updates every
colour once.  The colour of node (i, j, k) is (i + j + k) mod ncol; colours are
visited in ascending order, colour 0 ("red") first.  Two colours make the
7-point stencil's updates independent; the radius-two 13-point star needs three
colours (Sec. 2.1.2: 2 / 3 / 4 colours for 2nd / 4th / 6th order), with which a
node and all of its star neighbours at distance 1 and 2 differ in colour.

For one node p the Gauss-Seidel value solves (A phi)_p = f_p for phi_p:
phi_GS = phi_p + r_p / a_pp with r = f - A phi; SOR writes
phi_p + omega (phi_GS - phi_p).  Because nodes of one colour never couple, all
nodes of a colour may be updated from the same residual evaluation.

Eqs. 3-5: omega_opt = 2 / (1 + sqrt(1 - rJ^2)),
rJ = sum_a h_a^-2 cos(pi/N_a) / sum_a h_a^-2, omega_opt,a = 2 / (1 + pi/N).

Eq. omega_n (Chebyshev acceleration, Sec. 2.1.1): omega_0 = 1,
omega_1 = 1 / (1 - rJ^2 / 2), omega_{n+1} = 1 / (1 - rJ^2 omega_n / 4); the
paper starts the sequence from n = 1.  The paper cites the red-black scheme in
which the index advances once per colour pass (half sweep); that reading is
taken here: pass n of a solve (n = 1, 2, ... over colour passes) uses omega_n.
"""
from __future__ import annotations

import math

import numpy as np

from .grid import CartGrid
from .operators import diagonal, residual


def ncolours(order: int) -> int:
    return {2: 2, 4: 3}[order]


def colour_mask(grid: CartGrid, colour: int, ncol: int) -> np.ndarray:
    """Boolean mask over the interior: nodes with (i+j+k) mod ncol == colour."""
    I = grid.interior
    ix = grid.node_index(0)[I[2]]
    iy = grid.node_index(1)[I[1]]
    iz = grid.node_index(2)[I[0]]
    s = iz[:, None, None] + iy[None, :, None] + ix[None, None, :]
    return (s % ncol) == colour


def sweep_colour(phi: np.ndarray, f: np.ndarray, grid: CartGrid, colour: int, omega: float,
                 ncol: int | None = None) -> None:
    """SOR update of the nodes of one colour, in place on phi's interior."""
    if ncol is None:
        ncol = ncolours(grid.order)
    a_pp = diagonal(grid)
    I = grid.interior
    mask = colour_mask(grid, colour, ncol)
    r = residual(phi, f, grid)[I]
    inner = phi[I]
    inner[mask] += omega * r[mask] / a_pp
    phi[I] = inner


def sweep(phi: np.ndarray, f: np.ndarray, grid: CartGrid, omega: float = 1.0,
          ncol: int | None = None) -> None:
    """One full multicolour GS/SOR step, in place on phi's interior."""
    if ncol is None:
        ncol = ncolours(grid.order)
    for c in range(ncol):
        sweep_colour(phi, f, grid, c, omega, ncol)


def rjac_uniform(grid: CartGrid) -> float:
    """Eq. 4: Jacobi spectral radius estimate on a uniform Cartesian grid."""
    num = sum(math.cos(math.pi / grid.n[a]) / grid.h[a] ** 2 for a in range(3))
    den = sum(1.0 / grid.h[a] ** 2 for a in range(3))
    return num / den


def omega_opt(rj: float) -> float:
    """Eq. 3."""
    return 2.0 / (1.0 + math.sqrt(1.0 - rj * rj))


def omega_opt_a(n: int) -> float:
    """Eq. 5 (large-N approximation)."""
    return 2.0 / (1.0 + math.pi / n)


def omega_next(rj: float, omega_n: float) -> float:
    """Eq. omega_n: omega_{n+1} from omega_n."""
    return 1.0 / (1.0 - rj * rj * omega_n / 4.0)


def omega_first(rj: float) -> float:
    """Eq. omega_n: omega_1."""
    return 1.0 / (1.0 - rj * rj / 2.0)


def omega_sequence(rj: float, count: int) -> list:
    """omega_1 .. omega_count of Eq. omega_n (the sequence the paper uses)."""
    out = []
    w = omega_first(rj)
    for _ in range(count):
        out.append(w)
        w = omega_next(rj, w)
    return out

