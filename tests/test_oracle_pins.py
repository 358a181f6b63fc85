"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Every test here checks the oracle against something other than itself:
closed-form potentials, convergence orders under refinement, a dense direct
solve of an independently assembled matrix, textbook identities of the
transfer operators, brute-force sequential sweeps, library special functions,
the addition theorem, and the step counts printed in Table 3.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import krylov, multigrid, multipole as MP, smoothers as SM, solve as S
from oracle import spherical as SP, transfer as TR
from oracle.grid import cart_grid, hierarchy
from oracle.operators import laplacian, residual

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- operators

@pytest.mark.parametrize("order,expect,tol", [(2, 4.0, 0.3), (4, 16.0, 2.0)])
def test_manufactured_convergence_order(order, expect, tol):
    """sin(pi x) sin(pi y) sin(pi z): max error ratio under N -> 2N is 2^order."""
    errs = []
    for n in (16, 32, 64):
        rho, phi, exact = W.manufactured_sine(n, order)
        g = cart_grid(n, order)
        info = S.solve_cartesian(rho, phi, g, "mg", 1e-12)
        assert info.converged
        errs.append(np.max(np.abs(phi[g.interior] - exact[g.interior])))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    for r in ratios:
        assert abs(r - expect) < tol, ratios


def _lap1d(n, h, order):
    """1-D second-derivative matrix on interior nodes 1..n-1, zero boundary."""
    m = n - 1
    w = {2: [(-1, 1.0), (0, -2.0), (1, 1.0)],
         4: [(-2, -1 / 12), (-1, 16 / 12), (0, -30 / 12), (1, 16 / 12), (2, -1 / 12)]}[order]
    D = np.zeros((m, m))
    for i in range(m):
        for d, c in w:
            j = i + d
            if 0 <= j < m:
                D[i, j] += c / h ** 2
    return D


def _dense_matrix(n, order):
    h = 1.0 / n
    D = _lap1d(n, h, order)
    I = np.eye(n - 1)
    return (np.kron(I, np.kron(I, D)) + np.kron(I, np.kron(D, I)) + np.kron(D, np.kron(I, I)))


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("method", ["cg", "pcg", "mg", "sor", "ir"])
def test_dense_direct_solve(order, method):
    """8^3 intervals, zero boundary, random rho: iterative solutions agree with
    numpy.linalg.solve on a Kronecker-sum matrix assembled independently."""
    n = 8 if method != "mg" else 16        # MG needs one coarsening (>= 16)
    g = cart_grid(n, order)
    gen = W.rng(11)
    rho = np.zeros(g.shape)
    rho[g.interior] = gen.standard_normal(rho[g.interior].shape)
    A = _dense_matrix(n, order)
    x = np.linalg.solve(A, (4 * math.pi * rho[g.interior]).ravel())
    phi = g.zeros()
    kw = {"omega": 1.5} if method == "sor" else {}
    info = S.solve_cartesian(rho, phi, g, method, 1e-13, max_iter=20000, **kw)
    assert info.converged
    got = phi[g.interior].ravel()
    assert np.max(np.abs(got - x)) / np.max(np.abs(x)) < 1e-11


def test_operator_matches_dense_matrix():
    for order in (2, 4):
        n = 8
        g = cart_grid(n, order)
        v = g.zeros()
        v[g.interior] = W.rng(3).standard_normal(v[g.interior].shape)
        A = _dense_matrix(n, order)
        got = laplacian(v, g)[g.interior].ravel()
        np.testing.assert_allclose(got, A @ v[g.interior].ravel(), rtol=1e-13, atol=1e-9)


def test_uniform_sphere_closed_form():
    """Config with rho = 1 in a sphere of radius 0.25: error vs the textbook
    potential <= 2e-2 at N = 32 and decreasing under refinement."""
    errs = []
    for n in (16, 32):
        rho, phi, exact = W.uniform_sphere(n)
        g = cart_grid(n)
        S.solve_cartesian(rho, phi, g, "mg", 1e-10)
        I = g.interior
        errs.append(np.max(np.abs(phi[I] - exact[I])) / np.max(np.abs(exact[I])))
    assert errs[1] <= 2e-2
    assert errs[1] < errs[0]


def _phi_smooth_sphere(X, Y, Z, c, a, m, G=1.0):
    """Sec. 3.1 closed form (reading (x - x_p)^2 for the garbled (x - x_p^2))."""
    rp = m / (32 * math.pi * a ** 3 / 105)
    d = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    w = d / a
    inside = 4 * math.pi * G * rp * a ** 2 * (-1 / 6 + w ** 2 / 6 - w ** 4 / 10 + w ** 6 / 42)
    return np.where(d < a, inside, -G * m / np.maximum(d, 1e-300))


def test_smooth_sphere_closed_form_is_a_poisson_solution():
    """The printed potential satisfies Eq. 1 for the printed density (checked by
    centred differences of the closed form) and is continuous at d = a."""
    c, a, m = (0.1, -0.05, 0.02), 0.3, 1.5
    h = 1e-3
    pts = np.array([[0.1, -0.05, 0.1], [0.25, 0.0, 0.0], [0.5, 0.4, -0.3], [0.1, 0.1, 0.05]])
    for p in pts:
        lap = 0.0
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = h
            f = lambda q: _phi_smooth_sphere(*q, c, a, m)
            lap += (f(p + e) - 2 * f(p) + f(p - e)) / h ** 2
        d = np.linalg.norm(p - np.array(c))
        rho = m / (32 * math.pi * a ** 3 / 105) * (1 - (d / a) ** 2) ** 2 if d < a else 0.0
        assert abs(lap - 4 * math.pi * rho) < 1e-4 * max(1.0, 4 * math.pi * rho)
    inner = _phi_smooth_sphere(np.array(c[0] + a - 1e-12), np.array(c[1]), np.array(c[2]), c, a, m)
    assert abs(inner + m / a) < 1e-9


def test_smooth_sphere_second_order():
    """Dirichlet data from the closed form, one resolved sphere: error ~ h^2."""
    c, a, m = (0.0, 0.0, 0.0), 0.6, 1.0
    errs = []
    for n in (16, 32, 64):
        g = cart_grid(n, 2, (-1, -1, -1), (1, 1, 1))
        x, y, z = g.coords(0), g.coords(1), g.coords(2)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        exact = _phi_smooth_sphere(X, Y, Z, c, a, m)
        rho = W.smooth_sphere_density(n, 2, [c], [a], [m])
        phi = exact.copy()
        phi[g.interior] = 0.0
        S.solve_cartesian(rho, phi, g, "mg", 1e-12)
        errs.append(np.max(np.abs(phi - exact)))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


# ------------------------------------------------------------------ smoothers

def _bruteforce_sweep(phi, f, n, order, omega):
    """Sequential per-colour lexicographic sweep, one node at a time."""
    w = {2: {1: 1.0}, 4: {1: 16 / 12, 2: -1 / 12}}[order]
    w0 = {2: -2.0, 4: -30 / 12}[order]
    h2 = (1.0 / n) ** 2
    g = order // 2
    ncol = {2: 2, 4: 3}[order]
    for c in range(ncol):
        for k in range(1, n):
            for j in range(1, n):
                for i in range(1, n):
                    if (i + j + k) % ncol != c:
                        continue
                    K, J, Ii = k + g - 1, j + g - 1, i + g - 1
                    off = 0.0
                    for d, wd in w.items():
                        off += wd * (phi[K, J, Ii + d] + phi[K, J, Ii - d] + phi[K, J + d, Ii]
                                     + phi[K, J - d, Ii] + phi[K + d, J, Ii] + phi[K - d, J, Ii])
                    diag = 3 * w0
                    gs = (f[K, J, Ii] * h2 - off) / diag
                    phi[K, J, Ii] += omega * (gs - phi[K, J, Ii])


@pytest.mark.parametrize("order", [2, 4])
def test_sweep_equals_sequential_gauss_seidel(order):
    n = 6
    g = cart_grid(n, order)
    gen = W.rng(5)
    phi = gen.standard_normal(g.shape)
    f = gen.standard_normal(g.shape)
    a = phi.copy()
    b = phi.copy()
    SM.sweep(a, f, g, 1.3)
    _bruteforce_sweep(b, f, n, order, 1.3)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


def test_two_colours_are_not_enough_for_radius_two():
    """Sec. 2.1.1: with two colours, independence holds only for radius one:
    a 2-colour sweep of the 13-point stencil depends on node order."""
    n = 6
    g = cart_grid(n, 4)
    gen = W.rng(6)
    phi = gen.standard_normal(g.shape)
    f = gen.standard_normal(g.shape)
    vec = phi.copy()
    SM.sweep(vec, f, g, 1.0, ncol=2)
    seq = phi.copy()
    # sequential 2-colour sweep in lexicographic order
    w = {1: 16 / 12, 2: -1 / 12}
    for c in range(2):
        for k in range(1, n):
            for j in range(1, n):
                for i in range(1, n):
                    if (i + j + k) % 2 != c:
                        continue
                    K, J, I = k + 1, j + 1, i + 1
                    off = sum(wd * (seq[K, J, I + d] + seq[K, J, I - d] + seq[K, J + d, I]
                                    + seq[K, J - d, I] + seq[K + d, J, I] + seq[K - d, J, I])
                              for d, wd in w.items())
                    seq[K, J, I] = (f[K, J, I] / n ** 2 - off) / (-3 * 30 / 12)
    assert np.max(np.abs(vec - seq)) > 1e-6


def test_omega_formulas():
    """Eqs. 3-5: uniform cube gives rJ = cos(pi/N), omega_opt = 2/(1+sin(pi/N));
    omega_opt,a approaches omega_opt as N grows."""
    for n in (16, 32, 64, 512):
        g = cart_grid(n)
        rj = SM.rjac_uniform(g)
        assert abs(rj - math.cos(math.pi / n)) < 1e-15
        assert abs(SM.omega_opt(rj) - 2 / (1 + math.sin(math.pi / n))) < 1e-12
    d32 = abs(SM.omega_opt_a(32) - SM.omega_opt(math.cos(math.pi / 32)))
    d512 = abs(SM.omega_opt_a(512) - SM.omega_opt(math.cos(math.pi / 512)))
    assert d512 < d32 / 100
    # anisotropic spacing weights the cosines by h^-2
    g = cart_grid((16, 32, 64), lo=(0, 0, 0), hi=(1, 1, 1))
    num = sum(math.cos(math.pi / g.n[a]) / g.h[a] ** 2 for a in range(3))
    assert abs(SM.rjac_uniform(g) - num / sum(1 / g.h[a] ** 2 for a in range(3))) < 1e-15


def test_sor_optimal_omega_beats_gauss_seidel():
    rho, phi, _ = W.uniform_sphere(16)
    g = cart_grid(16)
    it_gs = S.solve_cartesian(rho, phi.copy(), g, "sor", 1e-8, omega=1.0).iterations
    w = SM.omega_opt(SM.rjac_uniform(g))
    it_sor = S.solve_cartesian(rho, phi.copy(), g, "sor", 1e-8, omega=w).iterations
    assert it_sor < it_gs / 3


# ------------------------------------------------------------------- transfer

def test_restriction_prolongation_adjoint_and_constants():
    fine = cart_grid(16)
    coarse = fine.coarsen()
    gen = W.rng(7)
    u = fine.zeros()
    u[fine.interior] = gen.standard_normal(u[fine.interior].shape)
    v = coarse.zeros()
    v[coarse.interior] = gen.standard_normal(v[coarse.interior].shape)
    lhs = 8.0 * np.sum(TR.restrict(u, fine, coarse) * v)
    rhs = np.sum(u * TR.prolong(v, coarse, fine))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    one = fine.zeros()
    one[fine.interior] = 1.0
    np.testing.assert_allclose(TR.restrict(one, fine, coarse)[coarse.interior], 1.0, rtol=1e-15)
    c1 = coarse.zeros()
    c1[coarse.interior] = 1.0
    pc = TR.prolong(c1, coarse, fine)
    # away from the boundary (where coarse boundary values are zero) P keeps constants
    np.testing.assert_allclose(pc[2:-2, 2:-2, 2:-2], 1.0, rtol=1e-15)


def test_full_weighting_of_quadratic():
    """1-D full weighting maps x^2 to x^2 + h^2/2 per axis."""
    fine = cart_grid(16)
    coarse = fine.coarsen()
    x = fine.coords(0)
    u = np.broadcast_to(x[None, None, :] ** 2, fine.shape).copy()
    rc = TR.restrict(u, fine, coarse)[coarse.interior]
    xc = coarse.coords(0)[coarse.interior[2]]
    h = fine.h[0]
    np.testing.assert_allclose(rc, np.broadcast_to(xc ** 2 + h ** 2 / 2, rc.shape), rtol=1e-13)


def test_prolongation_is_trilinear():
    fine = cart_grid(16)
    coarse = fine.coarsen()
    xc, yc, zc = coarse.coords(0), coarse.coords(1), coarse.coords(2)
    lin = lambda X, Y, Z: 1.0 + 2 * X - 3 * Y + 0.5 * Z + X * Y * Z
    Zc, Yc, Xc = np.meshgrid(zc, yc, xc, indexing="ij")
    vc = coarse.zeros()
    vc[coarse.interior] = lin(Xc, Yc, Zc)[coarse.interior]
    pf = TR.prolong(vc, coarse, fine)
    Zf, Yf, Xf = np.meshgrid(fine.coords(2), fine.coords(1), fine.coords(0), indexing="ij")
    # trilinear interpolation reproduces multilinear functions exactly inside the
    # region spanned by interior coarse nodes (fine nodes 2..N-2)
    sl = (slice(2, -2), slice(2, -2), slice(2, -2))
    np.testing.assert_allclose(pf[sl], lin(Xf, Yf, Zf)[sl], rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------------ multigrid

def test_mg_grid_independent_convergence():
    """Sec. 2.1.3: MG convergence does not depend on the grid spacing; the
    V-cycle count to 1e-6 stays within 3-7 (Sec. 4) and flat in N."""
    counts, rhos = [], []
    for n in (32, 64):
        rho = W.gaussian_blobs(n, seed=2)
        g = cart_grid(n)
        phi = g.zeros()
        info = S.solve_cartesian(rho, phi, g, "mg", 1e-6, bc="multipole", lmax=4)
        counts.append(info.iterations)
        rhos.append(info.rho_conv)
    assert all(3 <= c <= 7 for c in counts), counts
    assert abs(counts[0] - counts[1]) <= 1
    assert abs(rhos[0] - rhos[1]) < 0.25 * max(rhos)


def test_ir_reproduces_mg():
    """One V-cycle on the error equation per refinement step is the MG
    iteration itself (linear stationary iteration), in float64."""
    rho = W.gaussian_blobs(32, seed=2)
    g = cart_grid(32)
    a, b = g.zeros(), g.zeros()
    ia = S.solve_cartesian(rho, a, g, "mg", 1e-10, bc="multipole")
    ib = S.solve_cartesian(rho, b, g, "ir", 1e-10, bc="multipole")
    assert ia.iterations == ib.iterations
    assert np.max(np.abs(a - b)) / np.max(np.abs(a)) < 1e-12


def test_hierarchy_levels():
    assert [l.n[0] for l in hierarchy(cart_grid(256))] == [256, 128, 64, 32, 16, 8]
    assert [l.n[0] for l in hierarchy(cart_grid(96))] == [96, 48, 24, 12]
    assert [l.n[0] for l in hierarchy(cart_grid(512))][-1] == 8


# ------------------------------------------------------------------ Table 3

def _two_sphere(n):
    cfg = json.load(open(os.path.join(GOLDEN, "two_sphere_setup.json")))
    g = cart_grid(n, 2, (-1, -1, -1), (1, 1, 1))
    rho = W.smooth_sphere_density(n, 2, cfg["centres"], cfg["radii"], cfg["masses"])
    return g, rho


@pytest.mark.parametrize("method,slack", [("CG2", 0.05), ("SOR", 0.12)])
def test_table3_step_counts(method, slack):
    """Steps to the residual reductions of Table 3 at N = 64 (cold start,
    multipole boundary, SOR with omega_opt,a of Eq. 5)."""
    tab = json.load(open(os.path.join(GOLDEN, "table3_steps.json")))
    n = 64
    g, rho = _two_sphere(n)
    for row in tab["rows"]:
        if row["method"] != method or row["N"] != n:
            continue
        phi = g.zeros()
        if method == "CG2":
            info = S.solve_cartesian(rho, phi, g, "cg", row["reduction"], bc="multipole",
                                     lmax=4, origin=(0, 0, 0))
        else:
            info = S.solve_cartesian(rho, phi, g, "sor", row["reduction"], bc="multipole",
                                     lmax=4, origin=(0, 0, 0), omega=SM.omega_opt_a(n))
        assert abs(info.iterations - row["steps"]) <= slack * row["steps"], (row, info.iterations)


# ------------------------------------------------------------------ multipole

def test_multipole_matches_addition_theorem():
    """Eq. outer_multipole + Eq. outer_expansion equal the Legendre form
    -G sum rho dV sum_l r'^l/r^(l+1) P_l(cos gamma) (numpy's Legendre series)."""
    n = 12
    g = cart_grid(n)
    rho = W.gaussian_blobs(n, seed=4, nblobs=3)
    for lmax in (0, 3, 8):
        q = MP.moments_cartesian(rho, g, (0.5, 0.5, 0.5), lmax)
        pts = [(0.5, 0.1, -0.2), (-0.5, -0.5, 0.5), (0.3, -0.5, 0.45), (0.0, 0.0, 0.6)]
        direct = MP.direct_legendre_potential(rho, g, (0.5, 0.5, 0.5), lmax, 1.0, pts)
        pp = np.array(pts)
        exp = MP.potential_points(q, pp[:, 0], pp[:, 1], pp[:, 2], lmax, 1.0)
        np.testing.assert_allclose(exp, direct, rtol=1e-13)


def test_monopole_is_total_mass_and_odd_moments_vanish():
    n = 16
    g = cart_grid(n)
    rho = W.gaussian_blobs(n, blobs=[W.Blob((0.5, 0.5, 0.5), 0.1, 1.0)])
    q = MP.moments_cartesian(rho, g, (0.5, 0.5, 0.5), 6)
    assert abs(q[0] - rho[g.interior].sum() / n ** 3) < 1e-15
    for l in (1, 3, 5):
        for m in range(-l, l + 1):
            assert abs(q[MP.idx(l, m)]) < 1e-16
    # an off-centre blob has a dipole along its offset
    rho2 = W.gaussian_blobs(n, blobs=[W.Blob((0.5, 0.5, 0.7), 0.05, 1.0)])
    q2 = MP.moments_cartesian(rho2, g, (0.5, 0.5, 0.5), 1)
    assert q2[MP.idx(1, 0)] > 0 and abs(q2[MP.idx(1, 1)]) < 1e-15 and abs(q2[MP.idx(1, -1)]) < 1e-15
    np.testing.assert_allclose(q2[MP.idx(1, 0)] / q2[0], 0.2, rtol=1e-4)


def test_real_harmonics_against_scipy_and_orthonormality():
    sp = pytest.importorskip("scipy.special")
    lmax = 6
    gen = W.rng(9)
    th = gen.uniform(0, math.pi, 40)
    ph = gen.uniform(-math.pi, math.pi, 40)
    Y = MP.real_sph_harm(lmax, th, ph)
    if hasattr(sp, "sph_harm_y"):
        for l in range(lmax + 1):
            for m in range(0, l + 1):
                c = sp.sph_harm_y(l, m, th, ph)          # complex, Condon-Shortley phase
                cs = (-1) ** m
                if m == 0:
                    np.testing.assert_allclose(Y[MP.idx(l, 0)], c.real, atol=1e-13)
                else:
                    np.testing.assert_allclose(Y[MP.idx(l, m)], cs * math.sqrt(2) * c.real, atol=1e-13)
                    np.testing.assert_allclose(Y[MP.idx(l, -m)], cs * math.sqrt(2) * c.imag, atol=1e-13)
    # orthonormality by Gauss-Legendre x trapezoid quadrature (exact for these degrees)
    xg, wg = np.polynomial.legendre.leggauss(16)
    phs = np.arange(32) * 2 * math.pi / 32
    T, Pp = np.meshgrid(np.arccos(xg), phs, indexing="ij")
    W2 = wg[:, None] * (2 * math.pi / 32)
    Yq = MP.real_sph_harm(lmax, T, Pp)
    G = np.array([[np.sum(a * b * W2) for b in Yq] for a in Yq])
    np.testing.assert_allclose(G, np.eye(len(Yq)), atol=1e-12)


def test_multipole_boundary_converges_to_green_sum():
    """Paper's two-sphere setup: the truncated expansion approaches the direct
    Green's sum -G sum rho dV / |x - x'| on the faces as l_max grows."""
    cfg = json.load(open(os.path.join(GOLDEN, "two_sphere_setup.json")))
    n = 32
    g = cart_grid(n, 2, (-1, -1, -1), (1, 1, 1))
    rho = W.smooth_sphere_density(n, 2, cfg["centres"], cfg["radii"], cfg["masses"])
    I = g.interior
    Z, Y, X = np.meshgrid(g.coords(2), g.coords(1), g.coords(0), indexing="ij")
    src = np.stack([X[I], Y[I], Z[I]], -1).reshape(-1, 3)
    w = (rho[I] * g.h[0] ** 3).ravel()
    keep = w > 0
    src, w = src[keep], w[keep]
    pts = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.0, 0.0, -1.0], [1.0, 1.0, 1.0], [0.3, -1.0, 0.2]])
    green = np.array([-np.sum(w / np.linalg.norm(src - p, axis=1)) for p in pts])
    errs = []
    for lmax in (0, 2, 4, 8):
        q = MP.moments_cartesian(rho, g, (0, 0, 0), lmax)
        v = MP.potential_points(q, pts[:, 0], pts[:, 1], pts[:, 2], lmax, 1.0)
        errs.append(np.max(np.abs(v - green) / np.abs(green)))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    # truncation bound ~ (r'_max / r_min)^(lmax+1) with r'_max = 0.48, r_min = 1
    assert errs[3] < 0.48 ** 9
    assert errs[3] < errs[1] / 10


# ------------------------------------------------------------------ spherical

def _sph_exact(rr, rin, rout):
    return 4 * math.pi * (np.log(rr / rout) + rin / rr - rin / rout) - 4 * math.pi * (rout - rin) / rout


def test_spherical_radial_closed_form_second_order():
    """rho = r^-2 on r_in < r < r_out with Neumann at r_in: Gauss's law gives
    Phi = 4 pi [ln(r/r_out) + r_in/r - r_in/r_out] - 4 pi (r_out - r_in)/r_out."""
    errs = []
    for nr in (32, 64, 128):
        r, th, ph = W.spherical_coords(nr, 4, 8, 0.01, 1.0)
        rho = W.spherical_density(r, th, ph, with_angles=False)
        op = SP.SphericalOperator(r, th, ph)
        phi = np.zeros(op.shape)
        phi[:, :, -1] = -4 * math.pi * (r[-1] - r[0]) / MP.radial_extended(r)[-1]
        res = SP.bicgstab_solve(phi, 4 * math.pi * rho, op, 1e-12, 5000)
        assert res.converged
        ex = _sph_exact(r, r[0], r[-1])
        errs.append(np.max(np.abs(phi[1:-1, 1:-1, 1:-1] - ex[None, None, :])) / np.max(np.abs(ex)))
    assert 3.5 < errs[0] / errs[1] < 4.6 and 3.5 < errs[1] / errs[2] < 4.6, errs


def test_fp64_residual_floor_of_the_spherical_workload():
    """Why the 256 x 128 x 256 spherical workload stops at relative residual
    1e-8 and not 1e-10: no FP64 potential can have a much smaller residual.
    Storing the exact discrete solution x* in FP64 perturbs every unknown by
    its rounding error, |d_i| <= ulp(x_i)/2, and the residual of fl(x*) is
    then exactly -A d.  The pole and inner-radius coefficients of the
    spherical operator reach 1e11, so ||A d|| / ||b|| is about 5e-10 for
    rounding errors of that size (measured here with d uniform in
    +-ulp(x_i)/2 about the Gauss's-law potential of the r^-2 density, whose
    magnitude the angular factors change by under 20%): a floor 5 times above
    1e-10 and a fifth of 1e-8."""
    r, th, ph = W.spherical_coords(256, 128, 256, 0.01, 1.0)
    op = SP.SphericalOperator(r, th, ph)
    rho = W.spherical_density(r, th, ph)
    f = 4 * math.pi * rho
    U = (slice(1, -1), slice(1, -1), slice(1, -1))
    q = MP.moments_spherical(rho, r, th, ph, 6)
    bd = np.zeros(op.shape)
    bd[1:-1, 1:-1, -1] = MP.spherical_outer_ghost(q, r, th, ph, 6, 1.0)
    ref = float(np.linalg.norm(f[U] - op.apply(bd)))
    x = np.broadcast_to(_sph_exact(r, r[0], r[-1])[None, None, :], op.apply(bd).shape)
    rng = np.random.Generator(np.random.PCG64(11))
    d = np.zeros(op.shape)
    d[U] = np.spacing(x) * rng.uniform(-0.5, 0.5, x.shape)
    floor = float(np.linalg.norm(op.apply(d))) / ref
    assert 2e-10 < floor < 2e-9, floor


def test_spherical_operator_annihilates_harmonics():
    """x^2 - y^2 and 2z^2 - x^2 - y^2 are harmonic: the truncation error of the
    discrete operator on them falls as h^2."""
    vals = []
    for n in (16, 32, 64):
        r, th, ph = W.spherical_coords(n, n, 2 * n, 0.5, 1.5)
        op = SP.SphericalOperator(r, th, ph)
        re = MP.radial_extended(r)
        P = np.zeros(op.shape)
        R, T, F = re[None, None, :], th[None, :, None], ph[:, None, None]
        P[1:-1, 1:-1, :] = (R * np.sin(T)) ** 2 * np.cos(2 * F) + R ** 2 * (3 * np.cos(T) ** 2 - 1)
        vals.append(np.max(np.abs(op.apply(P)[:, :, 1:])))
    assert 3.5 < vals[0] / vals[1] < 4.5 and 3.5 < vals[1] / vals[2] < 4.5, vals


def test_bicgstab_matches_dense_solve():
    r, th, ph = W.spherical_coords(6, 6, 8, 0.1, 1.0)
    op = SP.SphericalOperator(r, th, ph)
    nunk = 6 * 6 * 8
    A = np.zeros((nunk, nunk))
    for c in range(nunk):
        e = np.zeros(op.shape)
        e[1:-1, 1:-1, 1:-1].flat[c] = 1.0
        A[:, c] = op.apply(e).ravel()
    assert np.max(np.abs(A - A.T)) > 1e-3          # not symmetric (hence BiCGSTAB)
    rho = W.spherical_density(r, th, ph)
    phi = np.zeros(op.shape)
    phi[:, :, -1] = -1.0
    f = 4 * math.pi * rho
    bd = np.zeros(op.shape)
    bd[:, :, -1] = -1.0
    b = f[1:-1, 1:-1, 1:-1].ravel() - op.apply(bd).ravel()
    x = np.linalg.solve(A, b)
    res = SP.bicgstab_solve(phi, f, op, 1e-13, 2000)
    assert res.converged
    np.testing.assert_allclose(phi[1:-1, 1:-1, 1:-1].ravel(), x, rtol=1e-10)


def test_bicgstab_restarts_through_an_exact_breakdown():
    """A 3x3 system on which rhat.r becomes exactly zero at the first step
    (rhat = r0 = (2,0,0), r1 = (0,-0.4,0.8)): without the restart rule the next
    beta is 0/0 and the iterate turns NaN; with it the method restarts from r1
    and reaches the dense solution."""
    A = np.array([[2.0, 1.0, 0.0], [0.0, 1.0, 2.0], [-1.0, -1.0, 1.0]])
    b = np.array([2.0, 0.0, 0.0])
    inv = 1.0 / np.diag(A)
    ref = float(np.linalg.norm(b))
    plain = krylov.bicgstab(lambda x: A @ x, inv, b, np.zeros(3), 1e-13, 20, ref, restart=False)
    assert not plain.converged and not np.all(np.isfinite(plain.x))
    res = krylov.bicgstab(lambda x: A @ x, inv, b, np.zeros(3), 1e-13, 20, ref)
    assert res.converged and res.iterations <= 6
    np.testing.assert_allclose(res.x, np.linalg.solve(A, b), rtol=0, atol=1e-12)


def _textbook_right_jacobi_bicgstab(K, inv, b, k):
    """k passes of van der Vorst's BiCGSTAB (Saad, Iterative Methods, Alg. 7.7)
    applied to the right-preconditioned system K u = b with K = A diag(inv),
    x = diag(inv) u, written from the textbook with the dense product K formed
    explicitly.  Returns x_k and the recursive residual norms ||r_0..r_k||."""
    u = np.zeros_like(b)
    r = b.copy()
    r0s = r.copy()
    p = r.copy()
    norms = [float(np.sqrt(r @ r))]
    for _ in range(k):
        Kp = K @ p
        a = (r @ r0s) / (Kp @ r0s)
        s = r - a * Kp
        Ks = K @ s
        w = (Ks @ s) / (Ks @ Ks)
        u = u + a * p + w * s
        r_new = s - w * Ks
        beta = ((r_new @ r0s) / (r @ r0s)) * (a / w)
        p = r_new + beta * (p - w * Kp)
        r = r_new
        norms.append(float(np.sqrt(r @ r)))
    return inv * u, norms


def test_bicgstab_without_replacement_is_the_textbook_iteration():
    """With residual replacement switched off (it fires only when the budget
    ends) the oracle's BiCGSTAB is van der Vorst's method: on a small
    non-symmetric, diagonally graded system its iterate after k passes and its
    recursive residual norms equal a textbook transcription of Saad's Alg. 7.7
    for K = A diag(A)^-1, pass for pass.  A wrong alpha, omega or beta (sign,
    index, operand) changes the iterates at the first or second pass."""
    rng = np.random.Generator(np.random.PCG64(7))
    n = 40
    A = rng.standard_normal((n, n)) * 0.35
    A += np.diag(rng.uniform(2.0, 12.0, n))
    assert np.max(np.abs(A - A.T)) > 0.1
    b = rng.standard_normal(n)
    inv = 1.0 / np.diag(A)
    K = A * inv[None, :]
    ref = float(np.linalg.norm(b))
    for k in range(1, 13):
        res = krylov.bicgstab(lambda v: A @ v, inv, b, np.zeros(n), 1e-30, k, ref, replace=0.0)
        xk, norms = _textbook_right_jacobi_bicgstab(K, inv, b, k)
        np.testing.assert_allclose(res.x, xk, rtol=0, atol=1e-11 * np.max(np.abs(xk)))
        # recursive norms of passes 1..k-1 (the last entry is the replaced, true residual)
        np.testing.assert_allclose(np.array(res.history[:k]) * ref, norms[:k], rtol=1e-9)
        true = float(np.linalg.norm(b - A @ xk))
        assert res.history[k] * ref == pytest.approx(true, rel=1e-6, abs=1e-13)
    # the iteration really converges on this system (the comparison is not of noise)
    assert norms[-1] < 1e-6 * norms[0]


def test_bicgstab_stops_on_the_true_residual():
    """On the graded log-r grid (48x24x48, r_in = 0.01) the recursively updated
    BiCGSTAB residual drifts from b - A x: stopping on it leaves a true
    residual of 2e-10 > 1e-10.  The returned iterate must meet the tolerance
    on the residual recomputed from scratch with the operator."""
    r, th, ph = W.spherical_coords(48, 24, 48, 0.01, 1.0)
    op = SP.SphericalOperator(r, th, ph)
    rho = W.spherical_density(r, th, ph)
    f = 4 * math.pi * rho
    P = np.zeros(op.shape)
    P[:, :, -1] = -1.0
    res = SP.bicgstab_solve(P, f, op, 1e-10, 5000)
    assert res.converged
    U = (slice(1, -1), slice(1, -1), slice(1, -1))
    bd = np.zeros(op.shape)
    bd[:, :, -1] = P[:, :, -1]
    true = np.linalg.norm(f[U] - op.apply(P)) / np.linalg.norm(f[U] - op.apply(bd))
    assert true <= 1e-10, true
    assert res.history[-1] == pytest.approx(true, rel=1e-6)


def test_spherical_multipole_monopole_is_mass():
    """rho = r^-2: q_00 = sum_i dr_i * 2 pi sum_j sin(theta_j) dtheta exactly, and
    the midpoint spacings telescope to (r_{N-1} + r_N - r_0 - r_{-1}) / 2; the
    angular midpoint sum tends to 4 pi.  Higher moments vanish by symmetry."""
    r, th, ph = W.spherical_coords(64, 16, 32, 0.01, 1.0)
    rho = W.spherical_density(r, th, ph, with_angles=False)
    q = MP.moments_spherical(rho, r, th, ph, 2)
    re = MP.radial_extended(r)
    radial = 0.5 * (re[-1] + re[-2] - re[1] - re[0])
    angular = 2 * math.pi * np.sum(np.sin(th)) * math.pi / th.size
    assert abs(q[0] - radial * angular) < 1e-13 * q[0]
    assert abs(angular - 4 * math.pi) < 4 * math.pi * (math.pi / 16) ** 2 / 8
    others = [q[MP.idx(l, m)] for l in (1, 2) for m in range(-l, l + 1) if (l, m) != (2, 0)]
    assert np.max(np.abs(others)) < 1e-12 * q[0]
    # q_20 is the midpoint-rule error of int P_2(cos t) sin t dt = 0: O(dtheta^2)
    r2, th2, ph2 = W.spherical_coords(64, 32, 32, 0.01, 1.0)
    q2 = MP.moments_spherical(W.spherical_density(r2, th2, ph2, with_angles=False), r2, th2, ph2, 2)
    assert 3.8 < q[MP.idx(2, 0)] / q2[MP.idx(2, 0)] < 4.2


# ------------------------------------------------------------------ inputs

def test_lognormal_generator_statistics():
    rho = W.lognormal_field(32, order=4, seed=3)
    core = rho[1:-2, 1:-2, 1:-2]                 # the periodic 32^3 block
    assert abs(np.std(np.log(core)) - 1.0) < 1e-12
    assert abs(np.mean(np.log(core)) + 0.5) < 1e-12
    np.testing.assert_array_equal(rho[1], rho[-2])   # node N repeats node 0


# ------------------------------------------------------------------ SOR schedules

def test_omega_sequence_is_chebyshev_and_tends_to_eq3():
    """Eq. omega_n: the recurrence equals the Chebyshev form
    omega_n = 2 T_n(1/rJ) / (rJ T_{n+1}(1/rJ)) (numpy's Chebyshev series), falls
    monotonically from omega_1 and tends to omega_opt of Eq. 3 from above."""
    from numpy.polynomial import chebyshev as Ch
    for rj in (0.5, 0.9, math.cos(math.pi / 16), math.cos(math.pi / 64)):
        seq = SM.omega_sequence(rj, 6000)
        x = 1.0 / rj
        for n in (1, 2, 3, 7, 20):
            tn = Ch.chebval(x, [0] * n + [1])
            tn1 = Ch.chebval(x, [0] * (n + 1) + [1])
            assert abs(seq[n - 1] - 2 * tn / (rj * tn1)) < 1e-12 * seq[n - 1]
        assert all(b <= a for a, b in zip(seq[:50], seq[1:51])) and seq[1] < seq[0]
        assert abs(seq[-1] - SM.omega_opt(rj)) < 1e-12
        assert min(seq) >= SM.omega_opt(rj) - 1e-14


def test_rjac_uniform_is_the_jacobi_spectral_radius():
    """Eq. 4 is the spectral radius of the Jacobi iteration I - D^-1 A of the
    7-point Dirichlet Laplacian: dense eigenvalues on an anisotropic grid."""
    n = (6, 8, 10)
    g = cart_grid(n, lo=(0, 0, 0), hi=(1.0, 0.7, 1.6))
    Ds = [_lap1d(n[a], g.h[a], 2) for a in range(3)]
    I = [np.eye(n[a] - 1) for a in range(3)]
    A = (np.kron(I[2], np.kron(I[1], Ds[0])) + np.kron(I[2], np.kron(Ds[1], I[0]))
         + np.kron(Ds[2], np.kron(I[1], I[0])))
    J = np.eye(A.shape[0]) - A / np.diag(A)[:, None]
    rho = np.max(np.abs(np.linalg.eigvals(J)))
    assert abs(rho - SM.rjac_uniform(g)) < 1e-12


def test_rjac_local_special_cases():
    """Eq. local_rjac: equal physical spacings and extents give cos(pi/N); a
    dominant phi term gives cos(pi/N_phi); with the metric factors omitted it is
    Eq. 4 of a Cartesian grid."""
    N = 24
    r, dt = 2.0, 0.1
    rj = SP.rjac_local(r * dt, r, dt, 1.0, dt, N, N, N)
    assert abs(rj - math.cos(math.pi / N)) < 1e-15
    rj = SP.rjac_local(1.0, 1.0, 1.0, 1e-6, 1.0, 10, 20, 40)
    assert abs(rj - math.cos(math.pi / 40)) < 1e-9
    g = cart_grid((16, 32, 64), lo=(0, 0, 0), hi=(1.0, 0.5, 2.0))
    rj = SP.rjac_local(g.h[0], 1.0, g.h[1], 1.0, g.h[2], 16, 32, 64)
    assert abs(rj - SM.rjac_uniform(g)) < 1e-15


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("schedule", ["chebyshev", "opt"])
def test_sor_schedules_reach_dense_solution(order, schedule):
    """Chebyshev and Eq. 3 weights converge to numpy.linalg.solve's solution and
    need fewer steps than Gauss-Seidel."""
    n = 8
    g = cart_grid(n, order)
    gen = W.rng(12)
    rho = np.zeros(g.shape)
    rho[g.interior] = gen.standard_normal(rho[g.interior].shape)
    x = np.linalg.solve(_dense_matrix(n, order), (4 * math.pi * rho[g.interior]).ravel())
    phi = g.zeros()
    info = S.solve_cartesian(rho, phi, g, "sor", 1e-13, max_iter=5000, sor_schedule=schedule)
    assert info.converged
    got = phi[g.interior].ravel()
    assert np.max(np.abs(got - x)) / np.max(np.abs(x)) < 1e-11
    gs = S.solve_cartesian(rho, g.zeros(), g, "sor", 1e-13, max_iter=5000, omega=1.0)
    assert info.iterations < gs.iterations


def _sph_dense(op):
    nunk = op.nr * op.nt * op.np_
    A = np.zeros((nunk, nunk))
    for c in range(nunk):
        e = np.zeros(op.shape)
        e[1:-1, 1:-1, 1:-1].flat[c] = 1.0
        A[:, c] = op.apply(e).ravel()
    return A


@pytest.mark.parametrize("schedule", ["chebyshev", "opt", "fixed"])
def test_spherical_sor_matches_dense_solve(schedule):
    r, th, ph = W.spherical_coords(6, 6, 8, 0.1, 1.0)
    op = SP.SphericalOperator(r, th, ph)
    A = _sph_dense(op)
    rho = W.spherical_density(r, th, ph)
    f = 4 * math.pi * rho
    bd = np.zeros(op.shape)
    bd[:, :, -1] = -1.0
    x = np.linalg.solve(A, f[1:-1, 1:-1, 1:-1].ravel() - op.apply(bd).ravel())
    phi = np.zeros(op.shape)
    phi[:, :, -1] = -1.0
    it, conv, hist = SP.sor_solve_spherical(phi, f, op, 1e-13, 20000, schedule, omega=1.0)
    assert conv
    np.testing.assert_allclose(phi[1:-1, 1:-1, 1:-1].ravel(), x, rtol=1e-10)


def test_spherical_colour_pass_is_sequential_gauss_seidel():
    """With omega = 1 one colour pass equals node-by-node Gauss-Seidel over the
    nodes of that colour in any order (the mirror and periodic ghosts couple
    only nodes of different colours): brute force with the dense matrix."""
    r, th, ph = W.spherical_coords(6, 4, 8, 0.2, 1.0)
    op = SP.SphericalOperator(r, th, ph)
    A = _sph_dense(op)
    gen = W.rng(5)
    f = np.zeros(op.shape)
    f[1:-1, 1:-1, 1:-1] = gen.standard_normal((8, 4, 6))
    P = np.zeros(op.shape)
    P[1:-1, 1:-1, 1:-1] = gen.standard_normal((8, 4, 6))
    x = P[1:-1, 1:-1, 1:-1].ravel().copy()      # zero outer ghost: L P = A x
    b = f[1:-1, 1:-1, 1:-1].ravel()
    k, j, i = np.unravel_index(np.arange(x.size), (8, 4, 6))
    for c in (0, 1):
        idx = np.nonzero((i + j + k) % 2 == c)[0]
        for p in gen.permutation(idx):
            x[p] += (b[p] - A[p] @ x) / A[p, p]
        SP.sor_colour(P, f, op, c, 1.0)
    np.testing.assert_allclose(P[1:-1, 1:-1, 1:-1].ravel(), x, rtol=1e-12, atol=1e-12)


def test_spherical_local_chebyshev_beats_gauss_seidel():
    r, th, ph = W.spherical_coords(16, 8, 16, 0.1, 1.0)
    op = SP.SphericalOperator(r, th, ph)
    rho = W.spherical_density(r, th, ph)
    f = 4 * math.pi * rho
    runs = {}
    for sched in ("chebyshev", "fixed"):
        phi = np.zeros(op.shape)
        phi[:, :, -1] = -1.0
        runs[sched] = SP.sor_solve_spherical(phi, f, op, 1e-8, 20000, sched, omega=1.0)[0]
    assert runs["chebyshev"] < runs["fixed"] / 2


# ------------------------------------------------------------------ preconditioned CG

@pytest.mark.parametrize("order", [2, 4])
def test_sgs_preconditioner_is_symmetric_gauss_seidel(order):
    """The colour passes apply (D + U)^-1 D (D + L)^-1 of -A_0 split in colour
    order (dense blocks from the independently assembled Kronecker sum), and
    that matrix is symmetric positive definite, as CG needs."""
    from oracle import multigrid as MG
    n = 6
    g = cart_grid(n, order)
    A = -_dense_matrix(n, order)
    ncol = {2: 2, 4: 3}[order]
    m = n - 1
    k, j, i = np.unravel_index(np.arange(m ** 3), (m, m, m))
    col = (i + j + k + 3) % ncol          # node index = array index + 1 per axis
    lower = col[:, None] > col[None, :]
    upper = col[:, None] < col[None, :]
    same = (col[:, None] == col[None, :]) & ~np.eye(m ** 3, dtype=bool)
    assert np.all(A[same] == 0.0)         # one colour never couples with itself
    D = np.diag(np.diag(A))
    L = np.where(lower, A, 0.0)
    U = np.where(upper, A, 0.0)
    Minv = np.linalg.solve(D + U, D @ np.linalg.inv(D + L))
    r = W.rng(21).standard_normal(m ** 3)
    z = MG.sgs_preconditioner(g)(r)
    np.testing.assert_allclose(z, Minv @ r, rtol=1e-12, atol=1e-14 * np.max(np.abs(z)))
    assert np.max(np.abs(Minv - Minv.T)) <= 1e-12 * np.max(np.abs(Minv))
    assert np.min(np.linalg.eigvalsh(0.5 * (Minv + Minv.T))) > 0.0


def test_pcg_needs_fewer_iterations_than_cg():
    rho, phi, _ = W.uniform_sphere(32)
    g = cart_grid(32)
    it_cg = S.solve_cartesian(rho, phi.copy(), g, "cg", 1e-10).iterations
    it_pcg = S.solve_cartesian(rho, phi.copy(), g, "pcg", 1e-10).iterations
    assert it_pcg < 0.7 * it_cg



# ------------------------------------------------------------------ compact stencils, SPAI, Galerkin
from oracle import compact as CP


def _manufactured_generic(n):
    g = cart_grid(n)
    Z, Y, X = np.meshgrid(g.coords(2), g.coords(1), g.coords(0), indexing="ij")
    u = np.exp(0.5 * X) * np.sin(2 * Y + 0.1) * np.cos(1.5 * Z + 0.3)
    return g, u, (0.25 - 4.0 - 2.25) * u


@pytest.mark.parametrize("order,sizes,lo,hi", [(2, (16, 32), 3.7, 4.3), (4, (16, 32), 14.5, 17.5),
                                              (6, (16, 32, 64), 50.0, 70.0)])
def test_compact_schemes_order_of_accuracy(order, sizes, lo, hi):
    """Sec. 2.1.3 compact stencils of order 2, 4, 6: the max error of the
    discrete solution against a smooth closed form falls by 2^order per halving
    of h (MG with SPAI smoothing to 1e-14)."""
    errs = []
    for n in sizes:
        g, u, f = _manufactured_generic(n)
        phi = u.copy()
        phi[g.interior] = 0.0
        it, conv, hist = CP.mg_solve(phi, f, g, order, 1e-14, 80)
        assert conv
        errs.append(np.max(np.abs(phi - u)[g.interior]))
    ratio = errs[-2] / errs[-1]
    assert lo <= ratio <= hi, (errs, ratio)


def test_lfa_smoothing_factors_reproduce_table1():
    """Table 1's mu from local Fourier analysis of I - omega M A with the printed
    coefficients (within their 4-digit rounding); for order 6 the garbled delta
    cell is replaced by the LFA-optimal value, which reproduces the printed mu."""
    for order, tol in ((2, 3e-3), (4, 1e-3), (6, 1e-3)):
        assert abs(CP.lfa_mu(order) - CP.TABLE1[order][5]) <= tol, (order, CP.lfa_mu(order))
    # mu is sensitive to delta: the printed (garbled) 0.0909 gives no smoother at all
    co = list(CP.TABLE1[6])
    co[4] = 0.0909
    assert CP.lfa_mu(6, coeffs=tuple(co)) > 1.0


def test_galerkin_operator_equals_dense_rap():
    """R A P assembled as dense matrices (full weighting, compact 4th-order A,
    trilinear P = 8 R^T) on an 8^3 grid: its row at a coarse interior node is
    the isotropic radius-one stencil `galerkin` returns, and it is symmetric."""
    from oracle.transfer import prolong, restrict
    n, h = 8, 1.0 / 8
    fine = cart_grid(n)
    coarse = fine.coarsen()
    nf, nc = (n - 1) ** 3, (n // 2 - 1) ** 3
    def cols(op, src_grid, m):
        out = []
        for c in range(m):
            e = src_grid.zeros()
            e[src_grid.interior].flat[c] = 1.0    # the interior slice is a view
            out.append(op(e))
        return np.array(out).T
    A = cols(lambda e: CP.apply27(e, fine, CP.L_WEIGHTS[4], 1 / h ** 2)[fine.interior].ravel(), fine, nf)
    P = cols(lambda e: prolong(e, coarse, fine)[fine.interior].ravel(), coarse, nc)
    R = cols(lambda e: restrict(e, fine, coarse)[coarse.interior].ravel(), fine, nf)
    RAP = R @ A @ P
    assert np.max(np.abs(RAP - RAP.T)) <= 1e-12 * np.max(np.abs(RAP))
    w, beyond, spread = CP.galerkin(CP.L_WEIGHTS[4], h)
    assert beyond == 0.0 and spread <= 1e-12 * abs(w[0])
    row = RAP[13].reshape(3, 3, 3)          # coarse node (2,2,2), the centre of 3^3 unknowns
    for idx in itertools.product(range(3), repeat=3):
        d = tuple(v - 1 for v in idx)
        assert abs(row[idx] - w[CP.offset_class(d)]) <= 1e-12 * abs(w[0])


def test_mg_spai_convergence_factor_matches_table2():
    """Eq. rho of V(1,1) cycles with SPAI smoothing and Galerkin coarse operators
    (64^3, cold start to 1e-10) against Table 2's nu = 1 column (511^3): within
    15% for orders 2, 4 and 6; more smoothing steps converge faster."""
    from oracle.multigrid import convergence_factor
    table = {2: 0.102, 4: 0.065, 6: 0.068}
    g = cart_grid(64)
    f = 4 * math.pi * W.gaussian_blobs(64, seed=2)
    for order, ref in table.items():
        rhos = []
        for nu in (1, 2):
            phi = g.zeros()
            it, conv, hist = CP.mg_solve(phi, f, g, order, 1e-10, 40, nu, nu)
            assert conv
            rhos.append(convergence_factor(hist))
        assert abs(rhos[0] - ref) <= 0.15 * ref, (order, rhos)
        assert rhos[1] < rhos[0]


def test_sixth_order_mg_cycles_match_table4_and_do_not_depend_on_depth():
    """Table 4's method (sixth-order compact stencil, SPAI V(nu,nu), Galerkin
    coarse operators, multipole l_max 4) on the two-sphere problem of Sec. 3.1
    at 63^3 unknowns, cold start to residual reduction 1e-6: the V-cycle counts
    lie within 2 of the printed ones (7, 4, 3 for nu = 1, 2, 3 on DGX and LUMI;
    nano5 prints 4 for nu = 3).  Table 2 quotes its factors for "seven coarse
    levels" (511^3 down to a 3^3 coarsest grid); coarsening to 3^3 instead of
    7^3 unknowns changes nothing here: the coarsest level is solved to
    relative accuracy 1e-2, well below the factor of one cycle."""
    import dataclasses
    from oracle import multigrid as MG
    n = 64
    lo, hi = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    g = cart_grid(n, 2, lo, hi)
    rho = W.smooth_sphere_density(n, 2, [(0.0, 0.0, 0.4), (0.0, 0.0, -0.2)], [0.08, 0.08], [1.0, 2.0])
    phi_b = g.zeros()
    q = MP.moments_cartesian(rho, g, (0.0, 0.0, 0.0), 4)
    MP.apply_cartesian_bc(phi_b, g, q, (0.0, 0.0, 0.0), 4, 1.0)
    f = 4 * math.pi * rho
    printed = {1: 7, 2: 4, 3: 3}
    rhos = {}
    for nu, cyc in printed.items():
        phi = phi_b.copy()
        it, conv, hist = CP.mg_solve(phi, f, g, 6, 1e-6, 40, nu, nu)
        assert conv and abs(it - cyc) <= 2, (nu, it, cyc)
        rhos[nu] = MG.convergence_factor(hist)
    assert rhos[1] > rhos[2] > rhos[3]

    def deeper(grid):
        levels = [grid]
        while all(v % 2 == 0 and v >= 8 for v in levels[-1].n):
            levels.append(dataclasses.replace(levels[-1], n=tuple(v // 2 for v in levels[-1].n)))
        return levels
    assert [L.n[0] for L in deeper(g)] == [64, 32, 16, 8, 4]
    orig = CP.hierarchy
    CP.hierarchy = deeper
    try:
        phi = phi_b.copy()
        it, conv, hist = CP.mg_solve(phi, f, g, 6, 1e-6, 40, 2, 2)
    finally:
        CP.hierarchy = orig
    assert conv
    assert abs(MG.convergence_factor(hist) - rhos[2]) <= 0.01 * rhos[2]


def test_compact_mg_matches_dense_solve():
    """16^3, zero boundary, random rho: the SPAI multigrid solution of the
    compact 6th-order system equals numpy.linalg.solve on the dense 27-point
    matrix with the same right-hand side."""
    n, h = 16, 1.0 / 16
    g = cart_grid(n)
    gen = W.rng(17)
    f = g.zeros()
    f[g.interior] = gen.standard_normal(f[g.interior].shape)
    m = (n - 1) ** 3
    A = np.zeros((m, m))
    for c in range(m):
        e = g.zeros()
        e[g.interior].flat[c] = 1.0
        A[:, c] = CP.apply27(e, g, CP.L_WEIGHTS[6], 1 / h ** 2)[g.interior].ravel()
    b = CP.compact_rhs(f, g, 6)[g.interior].ravel()
    x = np.linalg.solve(A, b)
    phi = g.zeros()
    it, conv, hist = CP.mg_solve(phi, f, g, 6, 1e-13, 60)
    assert conv
    assert np.max(np.abs(phi[g.interior].ravel() - x)) <= 1e-11 * np.max(np.abs(x))


# ------------------------------------------------------------------ inner multipole boundary (spherical)

def test_inner_expansion_matches_addition_theorem():
    """Eqs. inner_multipole / inner_expansion against the independent
    addition-theorem form -G sum rho dV sum_l r^l / r'^(l+1) P_l(cos gamma), for
    masses outside radius 0.5 and points inside radius 0.3."""
    gen = W.rng(23)
    n = 400
    d = gen.standard_normal((n, 3))
    src = d / np.linalg.norm(d, axis=1)[:, None] * gen.uniform(0.5, 1.0, n)[:, None]
    vals = gen.uniform(0.1, 1.0, n)
    pts = gen.standard_normal((12, 3))
    pts = pts / np.linalg.norm(pts, axis=1)[:, None] * gen.uniform(0.05, 0.3, 12)[:, None]
    lmax = 6
    qb = MP.inner_moments_points(vals, src[:, 0], src[:, 1], src[:, 2], lmax)
    got = MP.inner_potential_points(qb, pts[:, 0], pts[:, 1], pts[:, 2], lmax, 1.0)
    ref = MP.direct_legendre_inner(vals, src, lmax, 1.0, pts)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_inner_expansion_converges_to_green_sum():
    """Inside the innermost mass the truncated inner expansion approaches the
    direct Green's sum -G sum rho dV / |x - x'| as l_max grows."""
    gen = W.rng(24)
    c = np.array([0.0, 0.3, 0.6])
    src = c + 0.05 * gen.standard_normal((300, 3))
    vals = np.full(300, 1.0 / 300)
    pts = np.array([[0.05, 0.0, 0.0], [0.0, -0.1, 0.05], [0.08, 0.08, -0.08]])
    ref = np.array([-np.sum(vals / np.linalg.norm(src - p, axis=1)) for p in pts])
    errs = []
    for lmax in (1, 3, 6):
        qb = MP.inner_moments_points(vals, src[:, 0], src[:, 1], src[:, 2], lmax)
        got = MP.inner_potential_points(qb, pts[:, 0], pts[:, 1], pts[:, 2], lmax, 1.0)
        errs.append(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3, errs


def test_bicgstab_with_inner_dirichlet_ghost_matches_dense():
    r, th, ph = W.spherical_coords(6, 6, 8, 0.1, 1.0)
    op = SP.SphericalOperator(r, th, ph, inner="dirichlet")
    nunk = 6 * 6 * 8
    A = np.zeros((nunk, nunk))
    for c in range(nunk):
        e = np.zeros(op.shape)
        e[1:-1, 1:-1, 1:-1].flat[c] = 1.0
        A[:, c] = op.apply(e).ravel()
    gen = W.rng(25)
    rho = W.spherical_density(r, th, ph)
    f = 4 * math.pi * rho
    phi = np.zeros(op.shape)
    phi[:, :, -1] = -1.0
    phi[1:-1, 1:-1, 0] = gen.uniform(-3.0, -2.0, (8, 6))
    phi[0] = phi[8]
    phi[9] = phi[1]
    bd = phi.copy()
    bd[1:-1, 1:-1, 1:-1] = 0.0
    x = np.linalg.solve(A, f[1:-1, 1:-1, 1:-1].ravel() - op.apply(bd).ravel())
    res = SP.bicgstab_solve(phi, f, op, 1e-13, 2000)
    assert res.converged
    np.testing.assert_allclose(phi[1:-1, 1:-1, 1:-1].ravel(), x, rtol=1e-10)


def test_spherical_inner_multipole_shell_closed_form_second_order():
    """A smooth shell rho = sin^2(pi (r-a)/(b-a)) on a < r < b inside the grid,
    inner and outer multipole boundaries: the potential converges at second
    order in the radial spacing to -G [M(r)/r + 4 pi int_r^inf rho r' dr']
    (quadrature), the exact exterior/interior solution of a spherical shell."""
    from scipy.integrate import quad
    a, b, r_in, r_out = 0.3, 0.8, 0.2, 1.0
    rho_r = lambda x: math.sin(math.pi * (x - a) / (b - a)) ** 2 if a < x < b else 0.0
    def exact(x):
        m = 4 * math.pi * quad(lambda t: rho_r(t) * t * t, a, min(max(x, a), b), limit=200)[0]
        o = 4 * math.pi * quad(lambda t: rho_r(t) * t, max(min(x, b), a), b, limit=200)[0]
        return -(m / x + o)
    errs = []
    for nr, nt in ((32, 8), (64, 16)):   # the moments' theta quadrature is second order too
        r = r_in + (r_out - r_in) * (np.arange(nr) + 0.5) / nr
        th = (np.arange(nt) + 0.5) * math.pi / nt
        ph = 2 * math.pi * np.arange(8) / 8
        rho = np.zeros((10, nt + 2, nr + 2))
        rho[1:-1, 1:-1, 1:-1] = np.array([rho_r(x) for x in r])[None, None, :]
        phi = np.zeros(rho.shape)
        info = S.solve_spherical(rho, phi, r, th, ph, 1e-12, max_iter=4000, lmax=2, inner_bc="multipole")
        assert info.converged
        ex = np.array([exact(x) for x in r])
        errs.append(np.max(np.abs(phi[1:-1, 1:-1, 1:-1] - ex[None, None, :])) / np.max(np.abs(ex)))
    assert 3.0 <= errs[0] / errs[1] <= 5.0, errs
