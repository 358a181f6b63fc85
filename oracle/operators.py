"""Cartesian Laplacians and residuals (oracle).

Eq. 1 discretised on a uniform vertex-centred grid with spacings (hx,hy,hz):

* order 2, 7-point (stencil radius one, Sec. 2.1.1):
      (phi[i+1] - 2 phi[i] + phi[i-1]) / h^2 summed over the three axes;
* order 4, 13-point star (the naive radius-two 4th-order stencil Sec. 2.1.3
  contrasts with compact stencils):
      (-phi[i+2] + 16 phi[i+1] - 30 phi[i] + 16 phi[i-1] - phi[i-2]) / (12 h^2).

Values on boundary and ghost nodes are Dirichlet data.  All functions return
full-shape arrays that are zero outside the interior.
"""
from __future__ import annotations

import numpy as np

from .grid import CartGrid

# 1-D second-derivative weights for offsets 0, 1, 2 (symmetric)
WEIGHTS = {2: (-2.0, 1.0), 4: (-30.0 / 12.0, 16.0 / 12.0, -1.0 / 12.0)}


def _shift(a: np.ndarray, interior, axis: int, d: int):
    """View of `a` at interior positions shifted by d along grid axis (x=0)."""
    sl = list(interior)
    ax = 2 - axis                     # array axes are (z, y, x)
    s = sl[ax]
    sl[ax] = slice(s.start + d, s.stop + d)
    return a[tuple(sl)]


def laplacian(phi: np.ndarray, grid: CartGrid) -> np.ndarray:
    """A phi on interior nodes (full-shape result, zero elsewhere)."""
    w = WEIGHTS[grid.order]
    I = grid.interior
    out = np.zeros_like(phi)
    acc = np.zeros(phi[I].shape)
    for axis in range(3):
        inv_h2 = 1.0 / grid.h[axis] ** 2
        term = w[0] * phi[I]
        for d in range(1, len(w)):
            term = term + w[d] * (_shift(phi, I, axis, d) + _shift(phi, I, axis, -d))
        acc += term * inv_h2
    out[I] = acc
    return out


def diagonal(grid: CartGrid) -> float:
    """Coefficient of phi[p] in (A phi)[p]."""
    w0 = WEIGHTS[grid.order][0]
    return sum(w0 / grid.h[a] ** 2 for a in range(3))


def residual(phi: np.ndarray, f: np.ndarray, grid: CartGrid) -> np.ndarray:
    """r = f - A phi on interior nodes (zero elsewhere)."""
    r = -laplacian(phi, grid)
    I = grid.interior
    r[I] += f[I]
    return r


def norm2(v: np.ndarray, grid: CartGrid) -> float:
    """Euclidean norm over interior nodes."""
    return float(np.sqrt(np.sum(v[grid.interior] ** 2)))


def reference_norm(phi: np.ndarray, f: np.ndarray, grid: CartGrid) -> float:
    """|| f - A phi0 || where phi0 keeps the boundary data of phi and is zero
    inside: the denominator of every relative residual (boundary terms folded
    into the right-hand side)."""
    z = phi.copy()
    z[grid.interior] = 0.0
    return norm2(residual(z, f, grid), grid)
