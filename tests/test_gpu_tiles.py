"""The TMA tile kernels (fused two-colour sweep, fused residual + restriction)
against the per-colour / two-kernel path they replace, through the C ABI.

The fused red-black sweep evaluates every red node with the same operands and
arithmetic as the red colour pass (halo nodes included), and every black node
from those red values, so a whole multigrid solve must come out bit for bit the
same with the tile kernels on every level (tile_min_n = 16) and with them off
(tile_min_n = -1), in both mixed precisions and for both stencils (FP64 levels
never use the tile kernels, so the FP64 cases check that the setting is inert).  Grids are ragged
against the 64 x 8 sweep tile and the 32 x 8 / 32 x 4 coarse restriction tiles.
The default setting is also checked against the FP64 oracle (iteration count
and potential).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import solve as OS
from oracle.grid import cart_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_03563_gb300 as P
    P.capi.lib()
    return P


def _solve(pkg, n, order, hi, rho, prec, tile_min_n, bc="multipole"):
    rho_t = torch.from_numpy(rho).cuda()
    phi = torch.zeros_like(rho_t)
    with pkg.CartesianSolver(n, order, hi=hi, bc=bc, lmax=4) as s:
        info = s.solve(rho_t, phi, tol=1e-10, method="mg", prec=prec, max_iter=60,
                       inner_cycles=2, tile_min_n=tile_min_n)
    torch.cuda.synchronize()
    return info, phi.cpu().numpy()


CASES = [
    ((64, 64, 64), 2, (1.0, 1.0, 1.0)),
    ((96, 64, 32), 2, (1.0, 0.7, 0.45)),     # anisotropic spacing, non-cubic, ragged tiles
    ((64, 48, 80), 4, (1.0, 1.0, 1.0)),      # 13-point: fused restriction only
    ((96, 64, 32), 4, (1.0, 0.7, 0.45)),
]


@pytest.mark.parametrize("n,order,hi", CASES)
@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32", "mixed_bf16"])
def test_tiles_bitwise_equal(pkg, n, order, hi, prec):
    rho = np.abs(W.rng(4).standard_normal(W.cart_shape(n, order)))
    i_off, p_off = _solve(pkg, n, order, hi, rho, prec, -1)
    i_on, p_on = _solve(pkg, n, order, hi, rho, prec, 16)
    assert i_off.converged and i_on.converged
    assert i_on.iterations == i_off.iterations
    assert i_on.rel_residual == i_off.rel_residual
    assert np.array_equal(p_on, p_off), float(np.max(np.abs(p_on - p_off)))


@pytest.mark.parametrize("n,order", [(64, 2), (64, 4)])
def test_tiles_default_vs_oracle(pkg, n, order):
    """Default tile setting (finest 64^3 level tiled) against the FP64 oracle."""
    rho = W.gaussian_blobs(n, seed=2, order=order)
    g = cart_grid(n, order)
    phi_o = g.zeros()
    info_o = OS.solve_cartesian(rho, phi_o, g, "mg", 1e-10, bc="multipole", lmax=4)
    info, phi = _solve(pkg, (n, n, n), order, (1.0, 1.0, 1.0), rho, "fp64", 0)
    assert info.iterations == info_o.iterations
    err = np.max(np.abs(phi - phi_o)) / np.max(np.abs(phi_o))
    assert err <= 1e-10, err


@pytest.mark.parametrize("rtile", [1, 2, 3])
@pytest.mark.parametrize("prec", ["mixed_fp32", "mixed_bf16"])
def test_every_restriction_tile_is_bitwise_equal(pkg, rtile, prec):
    """Each compiled tile shape of the register-blocked residual + restriction
    (z-chunks marching up and down) gives the two-kernel path's coarse
    right-hand sides, hence the same solve bit for bit, on a grid ragged against
    every tile (96 x 64 x 32 fine: 48 x 32 x 16 coarse against 32 x 8/12/16)."""
    n, hi = (96, 64, 32), (1.0, 0.7, 0.45)
    rho = np.abs(W.rng(5).standard_normal(W.cart_shape(n, 2)))
    i_off, p_off = _solve(pkg, n, 2, hi, rho, prec, -1)
    rho_t = torch.from_numpy(rho).cuda()
    phi = torch.zeros_like(rho_t)
    with pkg.CartesianSolver(n, 2, hi=hi, bc="multipole", lmax=4) as s:
        s.set_tuning(prec, nu1=2, nu2=2, inner_cycles=2, tile_min_n=16, restrict_tile=rtile)
        s.profile(True)
        info = s.solve(rho_t, phi, tol=1e-10, method="mg", prec=prec, max_iter=60, tuned=True)
        prof = s.profile_read()
        s.profile(False)
    torch.cuda.synchronize()
    assert prof["resid_restrict_finest"]["variant"] == rtile
    assert info.converged and info.iterations == i_off.iterations
    assert np.array_equal(phi.cpu().numpy(), p_off)
