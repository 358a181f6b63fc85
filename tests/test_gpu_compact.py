"""Compact-stencil multigrid with SPAI smoothing and Galerkin coarse operators
(Sec. 2.1.3) through the C ABI against the FP64 oracle: equal V-cycle counts
and potentials within 1e-10 for orders 2, 4, 6, ragged sizes, V(1,1) to V(3,3),
the multipole boundary; argument errors before GPU work."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import solve as OS
from oracle.grid import cart_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_03563_gb300 as P
    P.capi.lib()
    return P


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _pair(pkg, n, order, rho, phi0, nu, bc="dirichlet"):
    g = cart_grid(n)
    phi_o = phi0.copy()
    info_o = OS.solve_cartesian(rho, phi_o, g, "mg", 1e-10, max_iter=60, bc=bc, lmax=4, nu1=nu, nu2=nu,
                                compact_order=order)
    phi_t = dev(phi0)
    with pkg.CartesianSolver(n, bc=bc, lmax=4) as s:
        info = s.solve(dev(rho), phi_t, tol=1e-10, method="mg", nu1=nu, nu2=nu, max_iter=60,
                       compact_order=order)
    return info, info_o, host(phi_t), phi_o


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("nu", [1, 3])
def test_compact_mg_matches_oracle(pkg, order, nu):
    rho = W.gaussian_blobs(32, seed=4)
    info, info_o, got, ref = _pair(pkg, 32, order, rho, np.zeros(W.cart_shape(32, 2)), nu)
    assert info.converged and info_o.converged
    assert info.iterations == info_o.iterations, (info.iterations, info_o.iterations)
    assert rel_err(got, ref) <= FP64_TOL
    assert abs(info.rel_residual - info_o.rel_residual) <= 1e-3 * info_o.rel_residual


def test_compact_mg_ragged_multipole_order6(pkg):
    """48^3 (levels 48, 24, 12: a 12^3 coarsest level, rows not multiples of the
    32 x 8 thread tile) with the multipole boundary and smooth nonzero boundary
    data on the Galerkin hierarchy."""
    rho = W.gaussian_blobs(48, seed=6)
    info, info_o, got, ref = _pair(pkg, 48, 6, rho, np.zeros(W.cart_shape(48, 2)), 2, bc="multipole")
    assert info.converged and info.iterations == info_o.iterations
    assert rel_err(got, ref) <= FP64_TOL


def test_compact_order6_accuracy_on_gpu(pkg):
    """The GPU solution of the 6th-order compact scheme converges at ~h^6 to a
    smooth closed form (error ratio between 32^3 and 64^3 near 64)."""
    errs = []
    for n in (32, 64):
        g = cart_grid(n)
        Z, Y, X = np.meshgrid(g.coords(2), g.coords(1), g.coords(0), indexing="ij")
        u = np.exp(0.5 * X) * np.sin(2 * Y + 0.1) * np.cos(1.5 * Z + 0.3)
        rho = (0.25 - 4.0 - 2.25) * u / (4 * math.pi)
        phi0 = u.copy()
        phi0[g.interior] = 0.0
        phi = dev(phi0)
        with pkg.CartesianSolver(n) as s:
            info = s.solve(dev(rho), phi, tol=1e-14, method="mg", nu1=3, nu2=3, max_iter=80,
                           compact_order=6)
        assert info.converged
        errs.append(np.max(np.abs(host(phi) - u)[g.interior]))
    assert 45.0 <= errs[0] / errs[1] <= 75.0, errs


def test_compact_rejects_bad_arguments(pkg):
    rho = dev(np.zeros(W.cart_shape(32, 2)))
    with pkg.CartesianSolver(32) as s:
        with pytest.raises(pkg.capi.PoissonError):
            s.solve(rho, dev(np.zeros(W.cart_shape(32, 2))), method="mg", compact_order=3)
        with pytest.raises(pkg.capi.PoissonError):
            s.solve(rho, dev(np.zeros(W.cart_shape(32, 2))), method="mg", compact_order=4, prec="mixed_bf16")
    with pkg.CartesianSolver(32, hi=(1.0, 2.0, 1.0)) as s:
        with pytest.raises(pkg.capi.PoissonError):
            s.solve(rho, dev(np.zeros(W.cart_shape(32, 2))), method="mg", compact_order=4)


@pytest.mark.parametrize("order", [4, 6])
def test_compact_fp32_refinement_matches_fp64(pkg, order):
    """FP64 refinement around FP32 inner compact V-cycles reaches the same
    tolerance; its potential agrees with the FP64 oracle's to 1e-7."""
    n = 48
    rho = W.gaussian_blobs(n, seed=8)
    g = cart_grid(n)
    phi_o = np.zeros(W.cart_shape(n, 2))
    info_o = OS.solve_cartesian(rho, phi_o, g, "mg", 1e-10, max_iter=60, bc="multipole", lmax=4, nu1=2,
                                nu2=2, compact_order=order)
    phi_t = dev(np.zeros(W.cart_shape(n, 2)))
    with pkg.CartesianSolver(n, bc="multipole", lmax=4) as s:
        info = s.solve(dev(rho), phi_t, tol=1e-10, method="mg", prec="mixed_fp32", nu1=2, nu2=2,
                       max_iter=60, inner_cycles=2, compact_order=order)
    assert info.converged and info.rel_residual <= 1e-10
    assert rel_err(host(phi_t), phi_o) <= 1e-7


def test_compact_fp32_refinement_odd_smoothing_count(pkg):
    """V(1,2) inner cycles: the out-of-place FP32 smoothing steps end in the
    second array on every level and are copied back; the refinement still
    agrees with the FP64 oracle's V(1,2) solution to 1e-7."""
    n = 40
    rho = W.gaussian_blobs(n, seed=9)
    g = cart_grid(n)
    phi_o = np.zeros(W.cart_shape(n, 2))
    info_o = OS.solve_cartesian(rho, phi_o, g, "mg", 1e-10, max_iter=60, bc="multipole", lmax=4, nu1=1,
                                nu2=2, compact_order=6)
    assert info_o.converged
    phi_t = dev(np.zeros(W.cart_shape(n, 2)))
    with pkg.CartesianSolver(n, bc="multipole", lmax=4) as s:
        info = s.solve(dev(rho), phi_t, tol=1e-10, method="mg", prec="mixed_fp32", nu1=1, nu2=2,
                       max_iter=60, inner_cycles=2, compact_order=6)
    assert info.converged and info.rel_residual <= 1e-10
    assert rel_err(host(phi_t), phi_o) <= 1e-7


def test_compact_fp32_refinement_after_other_solves_on_the_handle(pkg):
    """The second arrays of the FP32 levels are shared with the 7-point fused
    sweeps; a compact refinement after a 7-point mixed solve (and after a
    compact one) on the same handle gives bit-identical results to a fresh
    handle's."""
    n = 48
    rho = dev(W.gaussian_blobs(n, seed=10))
    kw = dict(tol=1e-10, method="mg", prec="mixed_fp32", nu1=2, nu2=2, max_iter=60, inner_cycles=2,
              compact_order=6)
    with pkg.CartesianSolver(n, bc="multipole", lmax=4) as fresh:
        ref = dev(np.zeros(W.cart_shape(n, 2)))
        fresh.solve(rho, ref, **kw)
    with pkg.CartesianSolver(n, bc="multipole", lmax=4) as s:
        other = dev(np.zeros(W.cart_shape(n, 2)))
        s.solve(rho, other, tol=1e-10, method="mg", prec="mixed_fp32", max_iter=60, inner_cycles=2)
        for _ in range(2):
            got = dev(np.zeros(W.cart_shape(n, 2)))
            info = s.solve(rho, got, **kw)
            assert info.converged
            assert torch.equal(got, ref)
