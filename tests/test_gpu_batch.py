"""Batched multigrid executor (poisson_batch_*) through the C ABI.

One graph launch advances every solve in the batch; the phase kernels walk
work lists that span grids of different sizes.  Checks:
  * each solve in a mixed-size batch matches a separate poisson_solve: equal
    iteration counts, potentials equal up to the rounding of the reductions
    (the batch's norm and coarsest-CG reductions group differently);
  * a solve's result is bit for bit the same alone in a batch and in a mix
    (its reductions only see its own tiles);
  * continuous batching: solves added while others are in flight, slots reused;
  * 13-point and mixed FP32 refinement batches; agreement with the FP64 oracle.
"""
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


def _rho(n, order, seed):
    return torch.from_numpy(W.gaussian_blobs(n, order, seed=seed)).cuda()


def _solo(pkg, n, order, rho, prec="fp64", tol=1e-10):
    phi = torch.zeros_like(rho)
    with pkg.CartesianSolver(n, order, bc="multipole", lmax=4) as s:
        info = s.solve(rho, phi, tol=tol, method="mg", prec=prec, max_iter=60, inner_cycles=2)
    torch.cuda.synchronize()
    return info, phi


def _run_batch(pkg, b, solvers, rhos, tols, step=2):
    """Add all solves, step until every slot is done; return (infos, phis) in order."""
    phis = [torch.zeros_like(r) for r in rhos]
    slots = [b.add(s, r, p, tol=t, max_iter=60) for s, r, p, t in zip(solvers, rhos, phis, tols)]
    for _ in range(200):
        st, _ = b.poll()
        if all(st[sl] != 0 for sl in slots):
            break
        b.step(step)
    infos = [b.remove(sl) for sl in slots]
    torch.cuda.synchronize()
    return infos, phis


def _relerr(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("order", [2, 4])
def test_batch_matches_separate_solves(pkg, order):
    sizes = [32, 64, 48, 96]
    rhos = [_rho(n, order, 10 + k) for k, n in enumerate(sizes)]
    solvers = [pkg.CartesianSolver(n, order, bc="multipole", lmax=4) for n in sizes]
    try:
        with pkg.Batch(8, max(sizes), order=order, prec="fp64") as b:
            infos, phis = _run_batch(pkg, b, solvers, rhos, [1e-10] * len(sizes))
    finally:
        for s in solvers:
            s.close()
    for n, rho, info, phi in zip(sizes, rhos, infos, phis):
        info_s, phi_s = _solo(pkg, n, order, rho)
        assert info.converged and info_s.converged
        assert info.iterations == info_s.iterations, (n, info.iterations, info_s.iterations)
        assert _relerr(phi, phi_s) <= 1e-12, (n, _relerr(phi, phi_s))
        assert abs(info.rel_residual - info_s.rel_residual) <= 1e-3 * info_s.rel_residual


def test_batch_result_independent_of_the_mix(pkg):
    n = 64
    rho = _rho(n, 2, 3)
    others = [(32, _rho(32, 2, 4)), (96, _rho(96, 2, 5)), (48, _rho(48, 2, 6))]
    s0 = pkg.CartesianSolver(n, bc="multipole", lmax=4)
    so = [pkg.CartesianSolver(m, bc="multipole", lmax=4) for m, _ in others]
    try:
        with pkg.Batch(4, 96) as b:
            (i_alone,), (p_alone,) = _run_batch(pkg, b, [s0], [rho], [1e-10])
            infos, phis = _run_batch(pkg, b, [s0] + so, [rho] + [r for _, r in others], [1e-10] * 4)
    finally:
        for s in [s0] + so:
            s.close()
    assert infos[0].iterations == i_alone.iterations
    assert torch.equal(phis[0], p_alone)


def test_batch_continuous_admission_and_slot_reuse(pkg):
    """Two slots; a third solve waits for a free slot and reuses it while the
    other is still running; every result matches its separate solve."""
    sizes = [32, 64, 32]
    tols = [1e-6, 1e-10, 1e-10]
    rhos = [_rho(n, 2, 20 + k) for k, n in enumerate(sizes)]
    solvers = [pkg.CartesianSolver(n, bc="multipole", lmax=4) for n in sizes]
    phis = [torch.zeros_like(r) for r in rhos]
    infos = {}
    try:
        with pkg.Batch(2, 64) as b:
            live = {b.add(solvers[0], rhos[0], phis[0], tol=tols[0]): 0,
                    b.add(solvers[1], rhos[1], phis[1], tol=tols[1]): 1}
            pending = [2]
            reused = False
            for _ in range(200):
                b.step(1)
                st, _ = b.poll()
                for sl in [sl for sl in live if st[sl] != 0]:
                    k = live.pop(sl)
                    infos[k] = b.remove(sl)
                    if pending:
                        j = pending.pop()
                        sl2 = b.add(solvers[j], rhos[j], phis[j], tol=tols[j])
                        reused = reused or sl2 == sl
                        live[sl2] = j
                if not live:
                    break
    finally:
        for s in solvers:
            s.close()
    torch.cuda.synchronize()
    assert reused and sorted(infos) == [0, 1, 2]
    for k, (n, rho) in enumerate(zip(sizes, rhos)):
        info_s, phi_s = _solo(pkg, n, 2, rho, tol=tols[k])
        assert infos[k].converged and infos[k].iterations == info_s.iterations
        assert _relerr(phis[k], phi_s) <= 1e-12


def test_batch_mixed_fp32(pkg):
    sizes = [32, 64]
    rhos = [_rho(n, 2, 30 + k) for k, n in enumerate(sizes)]
    solvers = [pkg.CartesianSolver(n, bc="multipole", lmax=4) for n in sizes]
    try:
        with pkg.Batch(4, 64, prec="mixed_fp32", inner_cycles=2) as b:
            infos, phis = _run_batch(pkg, b, solvers, rhos, [1e-10] * 2)
    finally:
        for s in solvers:
            s.close()
    for n, rho, info, phi in zip(sizes, rhos, infos, phis):
        _, phi64 = _solo(pkg, n, 2, rho)
        info_m, phi_m = _solo(pkg, n, 2, rho, prec="mixed_fp32")
        assert info.converged and info.rel_residual <= 1e-10
        assert info.iterations == info_m.iterations
        assert _relerr(phi, phi64) <= 1e-7
        assert _relerr(phi, phi_m) <= 1e-9


def test_batch_matches_oracle(pkg):
    n = 32
    rho_np = W.gaussian_blobs(n, seed=2)
    g = cart_grid(n)
    phi_o = g.zeros()
    info_o = OS.solve_cartesian(rho_np, phi_o, g, "mg", 1e-10, bc="multipole", lmax=4)
    s = pkg.CartesianSolver(n, bc="multipole", lmax=4)
    try:
        with pkg.Batch(2, 32) as b:
            (info,), (phi,) = _run_batch(pkg, b, [s], [torch.from_numpy(rho_np).cuda()], [1e-10])
    finally:
        s.close()
    assert info.iterations == info_o.iterations
    p = phi.cpu().numpy()
    assert np.max(np.abs(p - phi_o)) / np.max(np.abs(phi_o)) <= 1e-10


def test_batch_rejects_bad_arguments(pkg):
    with pytest.raises(pkg.capi.PoissonError):
        pkg.Batch(0, 64)
    with pytest.raises(pkg.capi.PoissonError):
        pkg.Batch(4, 64, prec="mixed_bf16")
    with pkg.Batch(1, 32) as b, pkg.CartesianSolver(64, bc="multipole") as big:
        rho = _rho(64, 2, 1)
        with pytest.raises(pkg.capi.PoissonError):
            b.add(big, rho, torch.zeros_like(rho))   # larger than max_n


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32"])
def test_handle_reused_between_batch_and_solo(pkg, prec):
    """A handle that solved on its own (its loop graph captured), then ran in a
    batch, then solves on its own again (poisson_solve and begin/step/end)
    gives the same potential every time: the batch leaves no buffer the
    handle's captured graphs point to changed or freed."""
    n = 128
    rho = _rho(n, 2, 41)
    other = _rho(64, 2, 42)
    with pkg.CartesianSolver(n, bc="multipole", lmax=4) as s, \
            pkg.CartesianSolver(64, bc="multipole", lmax=4) as s2:
        p1 = torch.zeros_like(rho)
        i1 = s.solve(rho, p1, tol=1e-10, method="mg", prec=prec, max_iter=60, inner_cycles=2)
        with pkg.Batch(2, n, prec=prec, inner_cycles=2) as b:
            (ib, _), (pb, _) = _run_batch(pkg, b, [s, s2], [rho, other], [1e-10, 1e-10])
        p2 = torch.zeros_like(rho)
        i2 = s.solve(rho, p2, tol=1e-10, method="mg", prec=prec, max_iter=60, inner_cycles=2)
        p3 = torch.zeros_like(rho)
        s.begin(rho, p3, tol=1e-10, method="mg", prec=prec, max_iter=60, inner_cycles=2)
        s.step(60)
        i3 = s.end()
        torch.cuda.synchronize()
    assert i1.converged and ib.converged and i2.converged and i3.converged
    assert i1.iterations == i2.iterations == i3.iterations
    # the batch's FP32 colour passes round differently from the solo tile kernels
    assert abs(ib.iterations - i1.iterations) <= (0 if prec == "fp64" else 1)
    assert torch.equal(p1, p2) and torch.equal(p1, p3)
    assert _relerr(pb, p1) <= (1e-12 if prec == "fp64" else 1e-9)
