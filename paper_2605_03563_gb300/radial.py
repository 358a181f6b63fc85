"""Zero-padded radial grids for the multipole boundaries of spherical grids.

Sec. 2.2 / Sec. 3.3: the multipole expansions are more accurate when no mass
lies near the radii where they are evaluated, so the grid of the potential is
extended inward and outward beyond the active range r_in < r < r_out, the
density is zero in the extensions, and the expansions are written at the
extended ends (here: on the ghost shells next to the first and last nodes).
The active range is logarithmic; the outer extension continues it; the inner
extension (where continuing the logarithmic grid would make the spacing
needlessly small) continues it smoothly with a fourth-order polynomial in the
node index that matches the logarithmic grid's value, first and second
derivative at r_in and reaches r_in_pad with a chosen end spacing.
"""
from __future__ import annotations

import math

import numpy as np


def padded_log_radii(r_in: float, r_out: float, n: int, n_pad_in: int = 20, n_pad_out: int = 20,
                     r_in_pad: float | None = None, end_spacing: float | None = None):
    """Node radii of a logarithmic grid of n nodes on [r_in, r_out] with n_pad_in
    inner and n_pad_out outer extension nodes.  Returns (r, active) where
    `active` is the boolean mask of the n logarithmic nodes (the density must be
    zero elsewhere).  r_in_pad defaults to r_in / 2; end_spacing (the node
    spacing at r_in_pad) defaults to the mean spacing of the inner extension."""
    if not (0.0 < r_in < r_out) or n < 3:
        raise ValueError("need 0 < r_in < r_out and n >= 3")
    q = (r_out / r_in) ** (1.0 / (n - 1))
    lq = math.log(q)
    i = np.arange(n, dtype=np.float64)
    core = r_in * q ** i
    core[0], core[-1] = r_in, r_out
    out = r_out * q ** np.arange(1, n_pad_out + 1, dtype=np.float64)
    inner = np.zeros(0)
    if n_pad_in > 0:
        rp = r_in / 2.0 if r_in_pad is None else float(r_in_pad)
        if not (0.0 < rp < r_in):
            raise ValueError("need 0 < r_in_pad < r_in")
        m = n_pad_in
        ds = (r_in - rp) / m if end_spacing is None else float(end_spacing)
        # r(s) = r_in + a1 s + a2 s^2 + a3 s^3 + a4 s^4 for s in [-m, 0]:
        # C2 join with r_in q^s at s = 0, r(-m) = rp, r'(-m) = ds
        a1, a2 = r_in * lq, r_in * lq * lq / 2.0
        A = np.array([[-m ** 3, m ** 4], [3.0 * m * m, -4.0 * m ** 3]])
        rhs = np.array([rp - r_in + a1 * m - a2 * m * m, ds - a1 + 2.0 * a2 * m])
        a3, a4 = np.linalg.solve(A, rhs)
        s = -np.arange(m, 0, -1, dtype=np.float64)
        inner = r_in + a1 * s + a2 * s * s + a3 * s ** 3 + a4 * s ** 4
        if not np.all(np.diff(np.concatenate([inner, [r_in]])) > 0.0):
            raise ValueError("the inner extension is not monotone; adjust n_pad_in, r_in_pad or end_spacing")
    r = np.concatenate([inner, core, out])
    active = np.zeros(r.size, dtype=bool)
    active[inner.size:inner.size + n] = True
    return r, active
