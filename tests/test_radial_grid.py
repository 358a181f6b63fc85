"""Zero-padded radial grid of Sec. 2.2 / Sec. 3.3 (host code): a logarithmic
active range, an outer extension continuing it and an inner extension by a
fourth-order polynomial that joins it with continuous value, slope and
curvature and ends at r_in_pad with the requested spacing."""
import math

import numpy as np
import pytest

from workloads import padded_log_radii


def test_padded_grid_structure_and_smooth_join():
    r_in, r_out, n = 6e13, 1.5e16, 560
    r, act = padded_log_radii(r_in, r_out, n, n_pad_in=20, n_pad_out=20)
    assert r.size == 600 and act.sum() == n and act[20] and not act[19] and act[579] and not act[580]
    assert r[20] == r_in and r[579] == r_out
    assert abs(r[0] - r_in / 2) <= 1e-12 * r_in
    assert np.all(np.diff(r) > 0)
    q = (r_out / r_in) ** (1 / (n - 1))
    np.testing.assert_allclose(r[580:], r_out * q ** np.arange(1, 21), rtol=1e-12)
    # no kink at r_in: the spacing changes across the join as smoothly as along the
    # logarithmic grid (a linear continuation to r_in / 2 would jump by a factor 2.5)
    d = np.diff(r)
    assert abs(d[20] / d[19] - q) <= 0.02


def test_padded_grid_end_spacing_and_errors():
    r, act = padded_log_radii(1.0, 100.0, 64, n_pad_in=10, n_pad_out=0, r_in_pad=0.6, end_spacing=0.03)
    assert abs(r[0] - 0.6) <= 1e-12 and abs((r[1] - r[0]) - 0.03) <= 0.01
    assert act.sum() == 64 and r[-1] == 100.0
    with pytest.raises(ValueError):
        padded_log_radii(1.0, 100.0, 64, r_in_pad=1.5)
    with pytest.raises(ValueError):   # an end spacing the extension cannot hold: not monotone
        padded_log_radii(1.0, 100.0, 64, n_pad_in=10, r_in_pad=0.6, end_spacing=1.0)
