"""The compact multigrid's level operators as the library builds them on the
host (poisson_compact_operators, no GPU): the compact L_h of order 2, 4, 6 on
the finest level, Galerkin products R A P below, Table 1's SPAI weights scaled
by h_l^2 -- against the oracle's own construction (oracle/compact.py), which
its pins tie to Taylor expansions, brute-force Galerkin products and the
paper's Table 2 convergence factors."""
import numpy as np
import pytest

from oracle import compact as OC
from oracle.grid import cart_grid, hierarchy


@pytest.fixture(scope="module")
def ops():
    from paper_2605_03563_gb300 import build as B
    B.build()
    from paper_2605_03563_gb300 import ops as O
    return O


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("n", [64, 96])
def test_level_operators_match_the_oracle(ops, order, n):
    g = cart_grid(n)
    levels = hierarchy(g)
    want = OC.level_operators(levels, order)
    a, m, om = ops.compact_operators(order, g.h[0], len(levels))
    for l, lev in enumerate(levels):
        ref = np.array(want[l])
        assert np.allclose(a[l], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max()), (order, l, a[l], ref)
        om_ref, m_ref = OC.spai_weights(order, lev.h[0])
        assert np.allclose(m[l], m_ref, rtol=1e-14, atol=0.0), (order, l)
        assert om[l] == om_ref


def test_galerkin_keeps_the_row_sum_zero(ops):
    """A constant is in the null space of every level operator (Galerkin with
    full weighting and trilinear prolongation preserves it): centre + 6 faces
    + 12 edges + 8 corners = 0."""
    for order in (2, 4, 6):
        a, _, _ = ops.compact_operators(order, 1.0 / 128, 5)
        for w in a:
            s = w[0] + 6 * w[1] + 12 * w[2] + 8 * w[3]
            assert abs(s) <= 1e-12 * abs(w[0]), (order, w, s)


def test_invalid_arguments(ops):
    from paper_2605_03563_gb300 import capi
    for args in ((3, 0.1, 2), (6, 0.0, 2), (6, -1.0, 2), (6, float("nan"), 2), (6, 0.1, 0), (6, 0.1, 31)):
        with pytest.raises(capi.PoissonError):
            ops.compact_operators(*args)
