"""Failure detection on the GPU without a fault: the bounded mbarrier wait of
the TMA tile kernels, made to run out on a barrier that nothing arrives at,
returns PS_ERR_TIMEOUT within its limit and leaves the context usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_03563_gb300 as P
    return P


def test_bounded_waits_run_out_and_report_a_timeout(pkg):
    from paper_2605_03563_gb300 import capi, ops
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    # a wait after an earlier failure: 1 ms limit
    st, ms = ops.probe_bounded_wait(False, out)
    assert st == capi.PS_ERR_TIMEOUT, (st, capi.lib().poisson_last_error())
    assert 1.0 <= ms < 100.0, ms
    assert b"ran out" in capi.lib().poisson_last_error()
    # a kernel's first wait: 2 s limit
    st, ms = ops.probe_bounded_wait(True, out)
    assert st == capi.PS_ERR_TIMEOUT
    assert 2000.0 <= ms < 4000.0, ms
    # the context is still usable: a small solve runs and converges
    import workloads as W
    rho = torch.from_numpy(W.gaussian_blobs(32, seed=2)).cuda()
    phi = torch.zeros_like(rho)
    with pkg.CartesianSolver(32, bc="multipole", lmax=4) as s:
        info = s.solve(rho, phi, tol=1e-10, method="mg", prec="mixed_fp32")
    assert info.converged and np.isfinite(float(phi.abs().max()))
