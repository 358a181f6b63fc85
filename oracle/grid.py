"""Grid conventions and the multigrid level hierarchy (oracle).

Vertex-centred Cartesian grids (Sec. 2.1.3: full weighting needs 2^N k - 1
unknowns per axis; Sec. 3.3: quantities live on vertices).  "N^3" means N
intervals per axis, nodes 0..N, interior unknowns 1..N-1.  A radius-g stencil
needs g-1 extra ghost layers outside the boundary node layer.

Coarsening (Sec. 2.1.3, geometric, h_c = 2 h) takes every other node and is
repeated while every axis has an even interval count >= 16; the last level is
the coarsest, solved by CG.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class CartGrid:
    n: tuple            # intervals (nx, ny, nz)
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    order: int = 2      # 2 -> 7-point, 4 -> 13-point

    @property
    def g(self) -> int:
        return self.order // 2

    @property
    def h(self) -> tuple:
        return tuple((self.hi[a] - self.lo[a]) / self.n[a] for a in range(3))

    @property
    def shape(self) -> tuple:
        g = self.g
        nx, ny, nz = self.n
        return (nz + 2 * g - 1, ny + 2 * g - 1, nx + 2 * g - 1)

    @property
    def interior(self):
        """Slices (z, y, x) selecting the interior unknowns."""
        g = self.g
        nx, ny, nz = self.n
        return (slice(g, g + nz - 1), slice(g, g + ny - 1), slice(g, g + nx - 1))

    def node_index(self, axis: int):
        """Global node index of every array position along `axis` (x=0)."""
        g = self.g
        return np.arange(-(g - 1), self.n[axis] + g)

    def coords(self, axis: int):
        return self.lo[axis] + self.node_index(axis) * self.h[axis]

    def zeros(self):
        return np.zeros(self.shape)

    def coarsen(self) -> "CartGrid":
        return replace(self, n=tuple(v // 2 for v in self.n))


def cart_grid(n, order=2, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> CartGrid:
    nn = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
    return CartGrid(nn, tuple(map(float, lo)), tuple(map(float, hi)), order)


def hierarchy(grid: CartGrid):
    """Levels finest first: halve while all interval counts are even and >= 16."""
    levels = [grid]
    while all(v % 2 == 0 and v >= 16 for v in levels[-1].n):
        levels.append(levels[-1].coarsen())
    return levels
