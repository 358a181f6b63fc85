"""Grid transfer operators (oracle), Sec. 2.1.3.

Restriction is full weighting, R = R1d (x) R1d (x) R1d with R1d = [1 2 1]/4,
on vertex-centred grids: coarse node I sits on fine node 2I and

    f_c[I] = sum_{d in {-1,0,1}^3} w(dx) w(dy) w(dz) r[2I + d],  w = (1,2,1)/4.

Prolongation is P = c R^T with c chosen so that P preserves constants.  Every
fine node receives R^T weights that sum to 1/8 (one coarse node with weight
(1/2)^3, two with (1/2)^2 (1/4), four with (1/2)(1/4)^2 or eight with
(1/4)^3), so c = 8, which is trilinear interpolation.  Both are written as the
literal sums over the 27 offsets; coarse boundary values are zero (the coarse
problem is the error equation).
"""
from __future__ import annotations

import itertools

import numpy as np

from .grid import CartGrid

W1D = {-1: 0.25, 0: 0.5, 1: 0.25}
P_SCALE = 8.0


def _fine_view(a: np.ndarray, fine: CartGrid, coarse: CartGrid, d):
    """View of fine array `a` at nodes 2I + d for all coarse interior I."""
    g = fine.g
    sl = []
    for ax in (2, 1, 0):                       # array order z, y, x
        nc = coarse.n[ax]
        start = 2 * 1 + d[ax] + (g - 1)        # node 2*1 + d  -> array index
        stop = 2 * (nc - 1) + d[ax] + (g - 1) + 1
        sl.append(slice(start, stop, 2))
    return a[tuple(sl)]


def restrict(r_fine: np.ndarray, fine: CartGrid, coarse: CartGrid) -> np.ndarray:
    """Full-weighting restriction of an interior fine field to the coarse grid."""
    out = coarse.zeros()
    acc = np.zeros(out[coarse.interior].shape)
    for d in itertools.product((-1, 0, 1), repeat=3):      # d = (dx, dy, dz)
        w = W1D[d[0]] * W1D[d[1]] * W1D[d[2]]
        acc += w * _fine_view(r_fine, fine, coarse, d)
    out[coarse.interior] = acc
    return out


def prolong(e_coarse: np.ndarray, coarse: CartGrid, fine: CartGrid) -> np.ndarray:
    """P e = 8 R^T e: scatter every coarse interior value to its 27 fine
    neighbours with the full-weighting weights times 8."""
    out = fine.zeros()
    ec = e_coarse[coarse.interior]
    for d in itertools.product((-1, 0, 1), repeat=3):
        w = P_SCALE * W1D[d[0]] * W1D[d[1]] * W1D[d[2]]
        view = _fine_view(out, fine, coarse, d)
        view += w * ec
    # only interior fine nodes receive corrections (boundary data stays fixed)
    mask = np.zeros(fine.shape, dtype=bool)
    mask[fine.interior] = True
    out[~mask] = 0.0
    return out
