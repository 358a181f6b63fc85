"""Autotuner for the multigrid cycle shape, the refinement inner loop and the
tile shapes of the fused red-black sweep and the fused residual + restriction.

For a grid size, stencil order, precision and tolerance it times whole solves
of a seeded Gaussian-mixture density (the serving workload's recipe) and keeps
the fastest time to tolerance:
  1. every candidate (nu1, nu2) x inner V-cycles per refinement step with the
     library's default tile;
  2. for the mixed precisions of the 7-point stencil, every compiled tile shape
     of the TMA-staged fused sweep (poisson_set_tuning's sweep_tile 1..4) with
     the winner of step 1 (the shapes give bitwise equal results, so only the
     time differs);
  3. with the winner of step 2, every tile shape of the register-blocked fused
     residual + restriction (restrict_tile 1..3; bitwise equal as well).
Each candidate runs through the handle's tuning (set_tuning + tuned=True), the
same path a tuned caller takes.  Results are cached in a JSON table keyed by
"n:order:prec:tol"; CartesianSolver.use_table and PoissonServer(tuning_table=)
install an entry on a handle.
"""
from __future__ import annotations

import json
import os
import statistics

DEFAULT_CANDIDATES = [(1, 1), (2, 1), (1, 2), (2, 2), (3, 3)]
SWEEP_TILES = (1, 2, 3, 4)
RESTRICT_TILES = (1, 2, 3)
TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_table.json")


def key(n, order, prec, tol) -> str:
    return f"{n}:{order}:{prec}:{tol:g}"


def load(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(table: dict, path: str = TABLE) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(n: int, order: int = 2, prec: str = "fp64", tol: float = 1e-10, device=None,
         cycles=DEFAULT_CANDIDATES, inners=None, tiles=None, restrict_tiles=None, reps: int = 3,
         seed: int = 2, lmax: int = 4):
    """Time every candidate and return the best settings with all timings."""
    import torch
    import workloads as W
    from . import CartesianSolver
    device = device or torch.device("cuda", torch.cuda.current_device())
    if inners is None:
        inners = (1,) if prec == "fp64" else (1, 2, 3)
    if tiles is None:
        tiles = SWEEP_TILES if (prec != "fp64" and order == 2) else ()
    if restrict_tiles is None:
        restrict_tiles = RESTRICT_TILES if (prec != "fp64" and order == 2) else ()
    rho = W.gaussian_blobs_device(n, W.gaussian_blob_params(seed), device, order=order)
    phi = torch.zeros_like(rho)
    trials = []
    with CartesianSolver(n, order, bc="multipole", lmax=lmax) as s:
        def run(nu1, nu2, inner, tile, rtile=0):
            s.set_tuning(prec, nu1, nu2, inner, 0, tile, rtile)
            times, info = [], None
            for r in range(reps + 1):
                phi.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                info = s.solve(rho, phi, tol=tol, method="mg", prec=prec, max_iter=200, tuned=True)
                b.record()
                torch.cuda.synchronize()
                if r > 0:
                    times.append(a.elapsed_time(b))
            if info.converged:
                trials.append({"nu1": nu1, "nu2": nu2, "inner": inner, "sweep_tile": tile,
                               "restrict_tile": rtile, "ms": statistics.median(times),
                               "iterations": info.iterations})
        for (nu1, nu2) in cycles:
            for inner in inners:
                run(nu1, nu2, inner, 0)
        if not trials:
            raise RuntimeError(f"no candidate converged for n={n} order={order} prec={prec} tol={tol:g}")
        best = min(trials, key=lambda t: t["ms"])
        for tile in tiles:
            run(best["nu1"], best["nu2"], best["inner"], tile)
        best = min(trials, key=lambda t: t["ms"])
        for rtile in restrict_tiles:
            run(best["nu1"], best["nu2"], best["inner"], best["sweep_tile"], rtile)
        s.clear_tuning(prec)
    best = min(trials, key=lambda t: t["ms"])
    return dict(best, tile_min_n=0, trials=trials)


def tune_table(sizes, order=2, prec="fp64", tol=1e-10, path: str = TABLE, **kw) -> dict:
    table = load(path)
    for n in sizes:
        table[key(n, order, prec, tol)] = tune(n, order, prec, tol, **kw)
    save(table, path)
    return table


def lookup(table: dict, n: int, order=2, prec="fp64", tol=1e-10):
    e = table.get(key(n, order, prec, tol))
    if not e:
        return {}
    return {"nu1": e["nu1"], "nu2": e["nu2"], "inner": e["inner"],
            "sweep_tile": e.get("sweep_tile", 0), "restrict_tile": e.get("restrict_tile", 0),
            "tile_min_n": e.get("tile_min_n", 0)}
