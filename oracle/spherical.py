"""Spherical-grid Laplacian and BiCGSTAB solve (oracle).

Eq. 2 discretised by direct finite differences in flux form on nodes
r_i (any increasing radii, here logarithmic), theta_j = (j+1/2) pi / Ntheta,
phi_k = 2 pi k / Nphi:

  (1/r_i^2) [ r_{i+1/2}^2 (P_{i+1}-P_i)/(r_{i+1}-r_i)
              - r_{i-1/2}^2 (P_i-P_{i-1})/(r_i-r_{i-1}) ] / ((r_{i+1}-r_{i-1})/2)
+ 1/(r_i^2 sin(t_j) dt^2) [ sin(t_{j+1/2}) (P_{j+1}-P_j) - sin(t_{j-1/2}) (P_j-P_{j-1}) ]
+ (P_{k+1} - 2 P_k + P_{k-1}) / (r_i^2 sin^2(t_j) dp^2)

with r_{i+-1/2} the arithmetic midpoints and sin(t_{-1/2}) = sin(t_{Nt-1/2}) = 0
at the poles (Sec. 2.2: angular boundaries follow the coordinate symmetries;
phi is periodic).  The operator is not symmetric, hence BiCGSTAB (Sec. 2.1.2).
Inner boundary: Neumann by a mirror ghost P_{-1} = P_1 at r_{-1} = 2 r_0 - r_1,
or Dirichlet data on that ghost shell (the inner multipole expansion).
Outer boundary: Dirichlet ghost at r_N (multipole potential or given data).

Layout: (Nphi+2, Ntheta+2, Nr+2), r fastest, node (i,j,k) at [k+1, j+1, i+1].
"""
from __future__ import annotations

import math

import numpy as np

from . import krylov
from .multipole import radial_extended


class SphericalOperator:
    """inner = "neumann": mirror ghost P_{-1} = P_1; "dirichlet": the inner ghost
    shell holds data (the inner multipole expansion of Sec. 2.2)."""

    def __init__(self, r, th, ph, inner: str = "neumann"):
        if inner not in ("neumann", "dirichlet"):
            raise ValueError(inner)
        self.inner = inner
        self.r = np.asarray(r, dtype=np.float64)
        self.th = np.asarray(th, dtype=np.float64)
        self.ph = np.asarray(ph, dtype=np.float64)
        self.nr, self.nt, self.np_ = self.r.size, self.th.size, self.ph.size
        self.re = radial_extended(self.r)
        self.dth = math.pi / self.nt
        self.dph = 2.0 * math.pi / self.np_
        j = np.arange(self.nt + 1)
        sf = np.sin(j * math.pi / self.nt)           # sin(theta_{j-1/2}) for j=0..Nt
        sf[0] = 0.0
        sf[-1] = 0.0
        self.sin_face = sf
        self.sin_c = np.sin(self.th)

    @property
    def shape(self):
        return (self.np_ + 2, self.nt + 2, self.nr + 2)

    def fill_ghosts(self, P: np.ndarray) -> None:
        """Inner mirror and periodic phi ghosts (outer ghost untouched)."""
        if self.inner == "neumann":
            P[:, :, 0] = P[:, :, 2]
        P[0, :, :] = P[self.np_, :, :]
        P[self.np_ + 1, :, :] = P[1, :, :]

    def apply(self, P: np.ndarray) -> np.ndarray:
        """L P on the unknown nodes, shape (Nphi, Ntheta, Nr)."""
        P = P.copy()
        self.fill_ghosts(P)
        re = self.re
        ri = re[1:-1]
        rp = 0.5 * (re[2:] + re[1:-1])       # r_{i+1/2}
        rm = 0.5 * (re[1:-1] + re[:-2])      # r_{i-1/2}
        C = P[1:-1, 1:-1, 1:-1]
        rad = (rp ** 2 * (P[1:-1, 1:-1, 2:] - C) / (re[2:] - ri)
               - rm ** 2 * (C - P[1:-1, 1:-1, :-2]) / (ri - re[:-2])) / (0.5 * (re[2:] - re[:-2]))
        rad = rad / ri ** 2
        sp = self.sin_face[1:][None, :, None]
        sm = self.sin_face[:-1][None, :, None]
        sc = self.sin_c[None, :, None]
        th = (sp * (P[1:-1, 2:, 1:-1] - C) - sm * (C - P[1:-1, :-2, 1:-1])) / (
            ri[None, None, :] ** 2 * sc * self.dth ** 2)
        ph = (P[2:, 1:-1, 1:-1] - 2.0 * C + P[:-2, 1:-1, 1:-1]) / (
            ri[None, None, :] ** 2 * sc ** 2 * self.dph ** 2)
        return rad + th + ph

    def diagonal(self) -> np.ndarray:
        re = self.re
        ri = re[1:-1]
        rp = 0.5 * (re[2:] + re[1:-1])
        rm = 0.5 * (re[1:-1] + re[:-2])
        drad = -(rp ** 2 / (re[2:] - ri) + rm ** 2 / (ri - re[:-2])) / (0.5 * (re[2:] - re[:-2])) / ri ** 2
        sp = self.sin_face[1:][None, :, None]
        sm = self.sin_face[:-1][None, :, None]
        sc = self.sin_c[None, :, None]
        dth = -(sp + sm) / (ri[None, None, :] ** 2 * sc * self.dth ** 2)
        dph = -2.0 / (ri[None, None, :] ** 2 * sc ** 2 * self.dph ** 2)
        d = drad[None, None, :] + dth + dph
        return np.broadcast_to(d, (self.np_, self.nt, self.nr)).copy()


def bicgstab_solve(Pfield: np.ndarray, f: np.ndarray, op: SphericalOperator, tol: float,
                   max_iter: int, dot=krylov.numpy_dot):
    """Solve L P = f (f on the ghosted layout) with right-Jacobi BiCGSTAB.

    The outer ghost of Pfield is Dirichlet data; unknown nodes hold the
    initial guess and receive the solution."""
    U = (slice(1, -1), slice(1, -1), slice(1, -1))
    shp = Pfield[U].shape

    def apply_hom(v):
        full = np.zeros(op.shape)
        full[U] = v.reshape(shp)
        return op.apply(full).ravel()

    bdry = np.zeros(op.shape)
    bdry[:, :, -1] = Pfield[:, :, -1]
    if op.inner == "dirichlet":
        bdry[:, :, 0] = Pfield[:, :, 0]
    b = (f[U] - op.apply(bdry)).ravel()
    ref = float(np.sqrt(b @ b))
    if ref == 0.0:
        ref = 1.0
    inv_diag = (1.0 / op.diagonal()).ravel()
    res = krylov.bicgstab(apply_hom, inv_diag, b, Pfield[U].ravel().copy(), tol, max_iter, ref,
                          dot=dot)
    Pfield[U] = res.x.reshape(shp)
    return res


# ------------------------------------------------------------------ red-black SOR
# Sec. 2.1.1: the spherical implementation is red-black SOR whose weights depend
# on position: the sequence of Eq. omega_n (from n = 1, one n per colour pass)
# is run per node with the local Jacobi spectral radius of Eq. local_rjac,
#   rJ = [cos(pi/Nr) dr^-2 + cos(pi/Nt) (r dt)^-2 + cos(pi/Np) (r sin t dp)^-2]
#        / [dr^-2 + (r dt)^-2 + (r sin t dp)^-2].
# Readings: N_r, N_theta, N_phi are the numbers of unknown nodes per axis; dr_i
# is the width the flux form divides by, (r_{i+1} - r_{i-1}) / 2 with the
# operator's ghost radii; dt and dp are the uniform angular spacings.  The
# colour of node (i, j, k) is (i + j + k) mod 2: the mirror ghost P_{-1} = P_1
# and the periodic ghosts (Nphi even) take their values from nodes of the other
# colour, so the nodes of one colour never couple.

def rjac_local(dr, r, dt, sin_t, dp, nr: int, nt: int, nph: int):
    """Eq. local_rjac for broadcastable arrays of the local spacings."""
    wr = 1.0 / np.asarray(dr, dtype=np.float64) ** 2
    wt = 1.0 / (np.asarray(r, dtype=np.float64) * dt) ** 2
    wp = 1.0 / (np.asarray(r, dtype=np.float64) * np.asarray(sin_t, dtype=np.float64) * dp) ** 2
    num = math.cos(math.pi / nr) * wr + math.cos(math.pi / nt) * wt + math.cos(math.pi / nph) * wp
    return num / (wr + wt + wp)


def local_rjac_table(op: SphericalOperator) -> np.ndarray:
    """rJ of every (theta_j, r_i), shape (Ntheta, Nr)."""
    re = op.re
    dr = 0.5 * (re[2:] - re[:-2])
    return rjac_local(dr[None, :], op.r[None, :], op.dth, op.sin_c[:, None], op.dph,
                      op.nr, op.nt, op.np_)


def sor_colour(P: np.ndarray, f: np.ndarray, op: SphericalOperator, colour: int, omega) -> None:
    """P += omega (f - L P) / diag on the unknown nodes of one colour (in place);
    omega is a scalar or an (Ntheta, Nr) array."""
    U = (slice(1, -1), slice(1, -1), slice(1, -1))
    r = f[U] - op.apply(P)
    k = np.arange(op.np_)[:, None, None]
    j = np.arange(op.nt)[None, :, None]
    i = np.arange(op.nr)[None, None, :]
    mask = ((i + j + k) % 2) == colour
    w = np.broadcast_to(np.asarray(omega, dtype=np.float64), (op.nt, op.nr))[None, :, :]
    inner = P[U]
    upd = w * r / op.diagonal()
    inner[mask] += upd[mask]
    P[U] = inner


def sor_solve_spherical(Pfield: np.ndarray, f: np.ndarray, op: SphericalOperator, tol: float,
                        max_iter: int, schedule: str = "chebyshev", omega: float = 1.0):
    """Red-black SOR steps until ||f - L P|| <= tol ||b||, b = f - L(boundary part
    of P) as for BiCGSTAB.  schedule: "fixed" (omega), "opt" (Eq. 3 with the local
    rJ) or "chebyshev" (Eq. omega_n with the local rJ).  Returns (steps,
    converged, relative-residual history)."""
    U = (slice(1, -1), slice(1, -1), slice(1, -1))
    bdry = np.zeros(op.shape)
    bdry[:, :, -1] = Pfield[:, :, -1]
    if op.inner == "dirichlet":
        bdry[:, :, 0] = Pfield[:, :, 0]
    b = f[U] - op.apply(bdry)
    ref = float(np.sqrt(np.sum(b * b)))
    if ref == 0.0:
        ref = 1.0
    rel = lambda: float(np.sqrt(np.sum((f[U] - op.apply(Pfield)) ** 2))) / ref
    hist = [rel()]
    if hist[-1] <= tol:
        return 0, True, hist
    rj = local_rjac_table(op)
    w = 1.0 / (1.0 - rj * rj / 2.0)             # omega_1
    wopt = 2.0 / (1.0 + np.sqrt(1.0 - rj * rj))  # Eq. 3
    for it in range(1, max_iter + 1):
        for c in (0, 1):
            if schedule == "chebyshev":
                sor_colour(Pfield, f, op, c, w)
                w = 1.0 / (1.0 - rj * rj * w / 4.0)
            elif schedule == "opt":
                sor_colour(Pfield, f, op, c, wopt)
            elif schedule == "fixed":
                sor_colour(Pfield, f, op, c, omega)
            else:
                raise ValueError(schedule)
        hist.append(rel())
        if hist[-1] <= tol:
            return it, True, hist
    return max_iter, False, hist

