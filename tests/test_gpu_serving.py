"""Continuous batching: every request's result is the same alone and in the mix.

A small stream with two grid sizes, two tolerances and warm-started sequences
is served once with up to 8 solves in flight and once strictly one at a time,
with the batched executor (one graph launch per tick for all solves) and with
per-request graphs on separate streams; each request's potential must match
bit for bit (well inside the 1e-10 FP64 tolerance), with equal iteration
counts, and the two executors agree to 1e-12.  Also: warm starts help, the HBM budget gates admission, the
autotuner returns a converged configuration.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_03563_gb300 as P
    P.capi.lib()
    return P


def _stream():
    return W.serving_stream(n_requests=24, rate_hz=1e4, seed=7, sizes=(32, 64),
                            seq_fraction=0.5, seq_len=4, step_shift=0.01)


def _serve(pkg, reqs, max_active, **kw):
    from paper_2605_03563_gb300.serving import PoissonServer
    srv = PoissonServer(torch.device("cuda", 0), max_active=max_active, **kw)
    try:
        res, stats = srv.run(reqs, realtime=False, keep_results=True)
        phis = {rid: p.clone() for rid, p in srv.final_phi.items()}
    finally:
        srv.close()
    return {r.rid: r for r in res}, phis, stats


@pytest.mark.parametrize("executor", ["batch", "streams", "hybrid"])
def test_results_identical_alone_and_in_the_mix(pkg, executor):
    reqs = _stream()
    kw = dict(executor=executor, max_n=64, batch_max_n=32)
    mix, phi_mix, st_mix = _serve(pkg, reqs, max_active=8, **kw)
    solo, phi_solo, st_solo = _serve(pkg, reqs, max_active=1, **kw)
    assert st_mix["peak_active"] > 1 and st_solo["peak_active"] == 1
    assert len(mix) == len(reqs) == len(solo)
    for rid, r in mix.items():
        assert r.status == 0 and solo[rid].status == 0
        assert r.iterations == solo[rid].iterations
        assert r.rel_residual <= r.tol
        assert torch.equal(phi_mix[rid], phi_solo[rid]), rid


def test_batch_and_stream_executors_agree(pkg):
    """The batched executor and the per-request graphs give the same iteration
    counts and potentials equal to 1e-12 (the reductions group differently)."""
    reqs = _stream()
    bat, phi_b, _ = _serve(pkg, reqs, max_active=8, executor="batch", max_n=64)
    stm, phi_s, _ = _serve(pkg, reqs, max_active=8, executor="streams")
    for rid, r in bat.items():
        assert r.iterations == stm[rid].iterations
        err = float((phi_b[rid] - phi_s[rid]).abs().max() / phi_s[rid].abs().max())
        assert err <= 1e-12, (rid, err)


def test_warm_starts_take_fewer_cycles(pkg):
    reqs = _stream()
    res, _, _ = _serve(pkg, reqs, max_active=8)
    warm = [r.iterations for r in res.values() if r.warm]
    first = [r.iterations for r in res.values() if r.seq_id >= 0 and r.seq_step == 0]
    assert warm and first
    assert np.mean(warm) < np.mean(first)


def test_hbm_budget_gates_admission(pkg):
    from paper_2605_03563_gb300.serving import PoissonServer
    reqs = [r for r in _stream() if r.seq_id < 0][:6]
    n = max(r.n for r in reqs)
    one = PoissonServer.field_bytes(n)
    srv = PoissonServer(torch.device("cuda", 0), hbm_budget_bytes=3 * one + pkg.workspace_bytes(n) + (n + 1) ** 3 * 8,
                        max_active=8)
    try:
        res, stats = srv.run(reqs, realtime=False)
        assert len(res) == len(reqs) and all(r.status == 0 for r in res)
        assert stats["peak_active"] < len(reqs)
    finally:
        srv.close()
    tiny = PoissonServer(torch.device("cuda", 0), hbm_budget_bytes=1024)
    with pytest.raises(RuntimeError, match="HBM budget"):
        tiny.run(reqs[:1], realtime=False)
    tiny.close()


def test_autotuner_picks_a_converged_configuration(pkg):
    from paper_2605_03563_gb300 import autotune
    best = autotune.tune(32, prec="mixed_fp32", tol=1e-8, reps=1, cycles=[(1, 1), (2, 2)], inners=(1, 2),
                         tiles=(1, 3), restrict_tiles=(1, 2))
    assert (best["nu1"], best["nu2"]) in [(1, 1), (2, 2)] and best["inner"] in (1, 2)
    assert best["sweep_tile"] in (0, 1, 3) and best["restrict_tile"] in (0, 1, 2)
    assert best["ms"] == min(t["ms"] for t in best["trials"])
    assert len(best["trials"]) == 8


def test_tuned_tile_changes_the_launched_sweep_and_not_the_result(pkg, tmp_path):
    """A tuning installed on the handle (directly, or from an autotuner table,
    also through the server) changes the fused sweep's launched tile shape
    -- the profiler reports the variant of the launches it timed -- and the
    cycle shape; the potential equals that of an untuned solve with the same
    cycle shape bit for bit (the tile shapes share their arithmetic)."""
    import workloads as W
    from paper_2605_03563_gb300 import autotune
    from paper_2605_03563_gb300.serving import PoissonServer
    n, tol = 64, 1e-10
    rho = torch.from_numpy(W.gaussian_blobs(n, seed=2)).cuda()
    with pkg.CartesianSolver(n, bc="multipole", lmax=4) as s:
        ref = torch.zeros_like(rho)
        s.profile(True)
        info0 = s.solve(rho, ref, tol=tol, prec="mixed_fp32", nu1=1, nu2=2, inner_cycles=2)
        prof0 = s.profile_read()
        assert prof0["sweep_fused_finest"]["variant"] == 1          # FP32 default: 4 rows x 4 warps
        assert prof0["resid_restrict_finest"]["variant"] == 3       # 3 coarse rows x 4 warps
        s.set_tuning("mixed_fp32", nu1=1, nu2=2, inner_cycles=2, sweep_tile=3, restrict_tile=2)
        assert s.get_tuning("mixed_fp32")["sweep_tile"] == 3
        assert s.get_tuning("mixed_fp32")["restrict_tile"] == 2
        phi = torch.zeros_like(rho)
        info = s.solve(rho, phi, tol=tol, prec="mixed_fp32", tuned=True)   # nu1/nu2/inner from the tuning
        prof = s.profile_read()
        s.profile(False)
        assert prof["sweep_fused_finest"]["variant"] == 3
        assert prof["resid_restrict_finest"]["variant"] == 2
        assert info.converged and info.iterations == info0.iterations
        assert info.inner_cycles == info0.inner_cycles
        assert torch.equal(phi, ref)
        # the same through the autotuner's table
        path = str(tmp_path / "table.json")
        entry = {"nu1": 1, "nu2": 2, "inner": 2, "sweep_tile": 4, "restrict_tile": 3, "tile_min_n": 0,
                 "ms": 1.0, "trials": []}
        autotune.save({autotune.key(n, 2, "mixed_fp32", tol): entry}, path)
        got = s.use_table("mixed_fp32", tol, path)
        assert got == {"nu1": 1, "nu2": 2, "inner_cycles": 2, "tile_min_n": 0, "sweep_tile": 4,
                       "restrict_tile": 3}
        assert s.use_table("mixed_fp32", 1e-6, path) is None and s.get_tuning("mixed_fp32") is None
        s.use_table("mixed_fp32", tol, path)
        s.profile(True)
        phi.zero_()
        s.solve(rho, phi, tol=tol, prec="mixed_fp32", tuned=True)
        prof = s.profile_read()
        assert prof["sweep_fused_finest"]["variant"] == 4 and prof["resid_restrict_finest"]["variant"] == 3
        s.profile(False)
        assert torch.equal(phi, ref)
    # the server starts a request of that size with the table's settings
    reqs = [W.ServingRequest(0, 0.0, n, tol, W.gaussian_blob_params(2))]
    srv = PoissonServer(torch.device("cuda"), prec="mixed_fp32", executor="streams", max_n=n,
                        tuning_table=path)
    results, _ = srv.run(reqs, realtime=False, keep_results=True)
    srv.close()
    assert results[0].status == 0 and results[0].iterations == info0.iterations
