"""SOR weight schedules (Sec. 2.1.1) through the C ABI against the FP64 oracle:
the Chebyshev sequence of Eq. omega_n and omega_opt of Eq. 3 with rJ of Eq. 4
on Cartesian grids, and red-black SOR on the spherical grid with weights per
node from the local rJ of Eq. local_rjac.  FP64: identical step counts and
potentials within 1e-10."""
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


@pytest.mark.parametrize("schedule", ["chebyshev", "optimal"])
@pytest.mark.parametrize("n,order", [(32, 2), (16, 4)])
def test_cartesian_sor_schedules_match_oracle(pkg, schedule, n, order):
    if order == 2:
        rho, phi0, _ = W.uniform_sphere(n)
    else:
        rho, phi0, _ = W.manufactured_sine(n, order)
    g = cart_grid(n, order)
    phi_o = phi0.copy()
    info_o = OS.solve_cartesian(rho, phi_o, g, "sor", 1e-10, max_iter=5000,
                                sor_schedule={"chebyshev": "chebyshev", "optimal": "opt"}[schedule])
    phi_t = dev(phi0)
    with pkg.CartesianSolver(n, order) as s:
        info = s.solve(dev(rho), phi_t, tol=1e-10, method="sor", max_iter=5000, sor_schedule=schedule)
    assert info.converged and info_o.converged
    assert info.iterations == info_o.iterations, (info.iterations, info_o.iterations)
    assert rel_err(host(phi_t), phi_o) <= FP64_TOL
    assert abs(info.rel_residual - info_o.rel_residual) <= 1e-3 * info_o.rel_residual


def test_chebyshev_needs_fewer_steps_than_fixed_optimal_start(pkg):
    """The sequence starts gently (omega_1 ~ 1/(1 - rJ^2/2)) and reaches the
    optimal weight; both schedules need far fewer steps than Gauss-Seidel."""
    rho, phi0, _ = W.uniform_sphere(32)
    its = {}
    with pkg.CartesianSolver(32) as s:
        for sched, om in (("chebyshev", 1.0), ("optimal", 1.0), ("fixed", 1.0)):
            phi = dev(phi0)
            its[sched] = s.solve(dev(rho), phi, tol=1e-10, method="sor", max_iter=20000, omega=om,
                                 sor_schedule=sched).iterations
    assert its["chebyshev"] < its["fixed"] / 5 and its["optimal"] < its["fixed"] / 5


@pytest.mark.parametrize("schedule,omega", [("chebyshev", 1.0), ("optimal", 1.0), ("fixed", 1.6)])
def test_spherical_sor_matches_oracle(pkg, schedule, omega):
    r, th, ph = W.spherical_coords(16, 8, 16, 0.1, 1.0)
    rho = W.spherical_density(r, th, ph)
    phi_o = np.zeros(rho.shape)
    info_o = OS.solve_spherical(rho, phi_o, r, th, ph, 1e-10, max_iter=20000, lmax=6, method="sor",
                                omega=omega, sor_schedule={"optimal": "opt"}.get(schedule, schedule))
    phi_t = dev(np.zeros(rho.shape))
    with pkg.SphericalSolver(r, th, ph, bc="multipole", lmax=6) as s:
        info = s.solve(dev(rho), phi_t, tol=1e-10, method="sor", omega=omega, sor_schedule=schedule,
                       max_iter=20000)
    assert info.converged and info_o.converged
    assert info.iterations == info_o.iterations, (info.iterations, info_o.iterations)
    U = (slice(1, -1), slice(1, -1), slice(1, -1))
    got = host(phi_t)
    assert rel_err(got[U], phi_o[U]) <= FP64_TOL


def test_spherical_sor_rejects_mixed_precision(pkg):
    r, th, ph = W.spherical_coords(8, 4, 8, 0.1, 1.0)
    rho = W.spherical_density(r, th, ph)
    with pkg.SphericalSolver(r, th, ph) as s:
        with pytest.raises(pkg.capi.PoissonError):
            s.solve(dev(rho), dev(np.zeros(rho.shape)), method="sor", prec="mixed_fp32")


# ------------------------------------------------------------------ preconditioned CG
@pytest.mark.parametrize("n,order", [(32, 2), (16, 4), (24, 2)])
def test_pcg_matches_oracle(pkg, n, order):
    """CG preconditioned by multicolour symmetric Gauss-Seidel (Sec. 2.1.2):
    iteration counts equal to the oracle's, potentials within 1e-10; ragged
    rows (24^3: 23 interior nodes, an odd count) exercise the colour blocks."""
    if order == 2 and n == 32:
        rho, phi0, _ = W.uniform_sphere(n)
    elif order == 2:
        rho = np.abs(W.rng(31).standard_normal(W.cart_shape(n, 2)))
        phi0 = np.zeros(W.cart_shape(n, 2))
    else:
        rho, phi0, _ = W.manufactured_sine(n, order)
    g = cart_grid(n, order)
    phi_o = phi0.copy()
    info_o = OS.solve_cartesian(rho, phi_o, g, "pcg", 1e-10, max_iter=5000)
    phi_t = dev(phi0)
    with pkg.CartesianSolver(n, order) as s:
        info = s.solve(dev(rho), phi_t, tol=1e-10, method="pcg", max_iter=5000)
        phi_c = dev(phi0)
        info_c = s.solve(dev(rho), phi_c, tol=1e-10, method="cg", max_iter=5000)
    assert info.converged and info_o.converged
    assert info.iterations == info_o.iterations, (info.iterations, info_o.iterations)
    assert rel_err(host(phi_t), phi_o) <= FP64_TOL
    assert info.iterations < info_c.iterations


# ------------------------------------------------------------------ inner multipole boundary
@pytest.mark.parametrize("method", ["bicgstab", "sor"])
def test_spherical_inner_multipole_matches_oracle(pkg, method):
    """Eqs. inner_multipole / inner_expansion on the inner ghost shell (Sec. 2.2)
    with the outer expansion, off-centre density: ghost values to 1e-12,
    potentials to 1e-10 against the oracle (both solved to 1e-12: two BiCGSTAB
    runs that stop at 1e-10 may differ by cond(A) * 1e-10)."""
    r, th, ph = W.spherical_coords(24, 12, 24, 0.1, 1.0)
    rho = W.spherical_density(r, th, ph)
    rho[1:-1, 1:-1, 1:-1] *= (1.0 + 0.5 * np.cos(ph)[:, None, None] * np.sin(th)[None, :, None])
    phi_o = np.zeros(rho.shape)
    info_o = OS.solve_spherical(rho, phi_o, r, th, ph, 1e-12, max_iter=20000, lmax=6, method=method,
                                inner_bc="multipole")
    phi_t = dev(np.zeros(rho.shape))
    with pkg.SphericalSolver(r, th, ph, bc="multipole", lmax=6, inner="multipole") as s:
        info = s.solve(dev(rho), phi_t, tol=1e-12, method=method, max_iter=20000)
    assert info.converged and info_o.converged
    got = host(phi_t)
    np.testing.assert_allclose(got[1:-1, 1:-1, 0], phi_o[1:-1, 1:-1, 0], rtol=1e-12)
    np.testing.assert_allclose(got[1:-1, 1:-1, -1], phi_o[1:-1, 1:-1, -1], rtol=1e-12)
    U = (slice(1, -1), slice(1, -1), slice(1, -1))
    assert rel_err(got[U], phi_o[U]) <= FP64_TOL
    if method == "sor":
        assert info.iterations == info_o.iterations
    # the inner expansion is not the mirror: the two boundaries give different potentials
    phi_n = dev(np.zeros(rho.shape))
    with pkg.SphericalSolver(r, th, ph, bc="multipole", lmax=6) as s:
        s.solve(dev(rho), phi_n, tol=1e-10, method=method, max_iter=20000)
    assert rel_err(host(phi_n)[U], got[U]) > 1e-4


def test_spherical_padded_grid_multipole_boundaries(pkg):
    """Sec. 2.2's zero padding: density only on the active logarithmic range,
    extensions inward (polynomial, to r_in/2) and outward (logarithmic), both
    expansions written at the extended ends; BiCGSTAB against the oracle."""
    from workloads import padded_log_radii
    r, active = padded_log_radii(0.1, 1.0, 24, n_pad_in=6, n_pad_out=6)
    th = (np.arange(8) + 0.5) * np.pi / 8
    ph = 2 * np.pi * np.arange(16) / 16
    rho = W.spherical_density(r, th, ph)
    rho[:, :, 1:-1][:, :, ~active] = 0.0
    phi_o = np.zeros(rho.shape)
    info_o = OS.solve_spherical(rho, phi_o, r, th, ph, 1e-12, max_iter=20000, lmax=6, inner_bc="multipole")
    phi_t = dev(np.zeros(rho.shape))
    with pkg.SphericalSolver(r, th, ph, bc="multipole", lmax=6, inner="multipole") as s:
        info = s.solve(dev(rho), phi_t, tol=1e-12, max_iter=20000)
    assert info.converged and info_o.converged
    got = host(phi_t)
    U = (slice(1, -1), slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(got[1:-1, 1:-1, 0], phi_o[1:-1, 1:-1, 0], rtol=1e-12)
    assert rel_err(got[U], phi_o[U]) <= FP64_TOL
