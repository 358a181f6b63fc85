"""Continuous-batching solve server on the C ABI.

Requests (Cartesian multigrid solves of different sizes) arrive over time.  A
request is admitted when a slot is free and its device memory (handle
workspace, density, potential) fits the HBM budget; admitted solves are then
advanced together, `cycles_per_step` iterations per tick, with one of two
executors:
  * "batch": the batched executor (poisson_batch_*): one CUDA-graph launch per
    tick advances every active solve; its phase kernels walk work lists
    spanning all the grids in flight;
  * "streams": every solve is started with poisson_solve_begin and advanced by
    its own loop-graph launch on its handle's stream (requests' kernels
    overlap on the GPU);
  * "hybrid" (default): grids with at most `batch_max_n` intervals per axis go
    into the batched executor (small grids are latency-bound and gain most from
    sharing launches), larger ones run as their own loop graphs.  On the
    2000-request stream (200/s, cubes 32..256) this gave the lowest latencies:
    FP64 p50 177 ms (per-request graphs 235 ms, all in the batch 396 ms).
After each tick the server polls, ends finished solves, frees their slots and
admits new arrivals.  Handles (multigrid hierarchies and their
captured graphs) are cached per grid size and reused.  Members of a sequence
(consecutive steps of a slowly moving density) start from the previous step's
potential, kept on the device.  Each request's kernels and reductions are those
of a solo solve, so results do not depend on what else is in flight.
"""
from __future__ import annotations

import collections
import statistics
import time
from dataclasses import dataclass, field

from . import Batch, CartesianSolver, workspace_bytes


@dataclass
class Result:
    rid: int
    n: int
    tol: float
    arrival_s: float
    admit_s: float
    done_s: float
    iterations: int
    rel_residual: float
    status: int
    seq_id: int = -1
    seq_step: int = 0
    warm: bool = False

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


@dataclass
class _Slot:
    req: object
    solver: CartesianSolver
    rho: object
    phi: object
    admit_s: float
    warm: bool
    nbytes: int
    bslot: int = -1


class HandlePool:
    """Idle solver handles per grid size, with their device bytes."""

    def __init__(self, prec: str, lmax: int):
        self.prec, self.lmax = prec, lmax
        self.idle = collections.defaultdict(list)
        self.bytes_of = {}

    def handle_bytes(self, n: int) -> int:
        if n not in self.bytes_of:
            self.bytes_of[n] = workspace_bytes(n, 2, self.lmax, self.prec) + (n + 1) ** 3 * 8
        return self.bytes_of[n]

    def get(self, n: int):
        if self.idle[n]:
            return self.idle[n].pop(), False
        return CartesianSolver(n, bc="multipole", lmax=self.lmax), True

    def put(self, n: int, s: CartesianSolver):
        self.idle[n].append(s)

    def evict_one(self, keep: int = -1) -> int:
        """Free one idle handle (largest first, never of size `keep`); returns the
        bytes released."""
        for n in sorted(self.idle, reverse=True):
            if self.idle[n] and n != keep:
                self.idle[n].pop().close()
                return self.handle_bytes(n)
        return 0

    def close(self):
        for lst in self.idle.values():
            for s in lst:
                s.close()
        self.idle.clear()


class PoissonServer:
    def __init__(self, device, hbm_budget_bytes: int = 64 << 30, prec: str = "fp64",
                 cycles_per_step: int = 2, max_active: int = 64, lmax: int = 4, nu=(2, 2),
                 inner_cycles: int = 1, max_iter: int = 100, tuning: dict | None = None,
                 executor: str = "hybrid", max_n: int = 256, batch_max_n: int = 96,
                 tuning_table: dict | str | None = None):
        if executor not in ("batch", "streams", "hybrid"):
            raise ValueError("executor must be 'batch', 'streams' or 'hybrid'")
        self.device = device
        self.budget = int(hbm_budget_bytes)
        self.prec = prec
        self.k = int(cycles_per_step)
        self.max_active = int(max_active)
        self.lmax = lmax
        self.nu = nu
        self.inner = inner_cycles
        self.max_iter = max_iter
        self.tuning = tuning or {}
        # the autotuner's table ("n:order:prec:tol" -> settings incl. the fused
        # sweep's tile shape): requests that run on their own handle's loop graph
        # are started with the tuned settings of their size and tolerance
        if isinstance(tuning_table, str):
            from .autotune import load
            tuning_table = load(tuning_table)
        self.tuning_table = tuning_table
        self.pool = HandlePool(prec, lmax)
        self.used = 0                  # bytes held by handles (idle or busy), fields and warm potentials
        self.warm = {}                 # seq_id -> (phi tensor, step) of the last finished step
        self.final_phi = {}            # rid -> potential (when keep_results)
        self.executor = executor
        self.batch = None
        self.batch_max_n = max_n if executor == "batch" else (batch_max_n if executor == "hybrid" else 0)
        if self.batch_max_n > 0:
            # one (nu1, nu2, inner) for every grid of the batch
            self.batch = Batch(self.max_active, max(16, self.batch_max_n), order=2, prec=prec, nu1=nu[0],
                               nu2=nu[1], inner_cycles=inner_cycles)

    # ------------------------------------------------------------------ memory
    @staticmethod
    def field_bytes(n: int) -> int:
        return 2 * (n + 1) ** 3 * 8    # density + potential

    def _reserve(self, nbytes: int, keep: int = -1) -> bool:
        while self.used + nbytes > self.budget:
            freed = self.pool.evict_one(keep)
            if freed == 0:
                return False
            self.used -= freed
        self.used += nbytes
        return True

    def _settings(self, n: int):
        t = self.tuning.get(n, {})
        return (t.get("nu1", self.nu[0]), t.get("nu2", self.nu[1]), t.get("inner", self.inner))

    # ------------------------------------------------------------------ admission
    def _admissible(self, req) -> bool:
        if req.seq_id < 0 or req.seq_step == 0:
            return True
        w = self.warm.get(req.seq_id)
        return w is not None and w[1] == req.seq_step - 1

    def _admit(self, req, now: float):
        import torch
        from workloads import gaussian_blobs_device
        n = req.n
        need = self.field_bytes(n)
        fresh = not self.pool.idle[n]
        if fresh:
            need += self.pool.handle_bytes(n)
        if not self._reserve(need, keep=n):
            return None
        solver, created = self.pool.get(n)
        rho = gaussian_blobs_device(n, req.blobs, self.device, shift=req.shift)
        warm = False
        if req.seq_id >= 0 and req.seq_step > 0:
            phi, _ = self.warm.pop(req.seq_id)
            self.used -= (n + 1) ** 3 * 8
            warm = True
        else:
            phi = torch.zeros_like(rho)
        slot = _Slot(req, solver, rho, phi, now, warm, self.field_bytes(n) + (self.pool.handle_bytes(n) if fresh else 0))
        if self.batch is not None and n <= self.batch_max_n:
            slot.bslot = self.batch.add(solver, rho, phi, tol=req.tol, max_iter=self.max_iter)
        elif self.tuning_table is not None and solver.use_table(self.prec, req.tol, self.tuning_table):
            solver.begin(rho, phi, tol=req.tol, method="mg", prec=self.prec, max_iter=self.max_iter,
                         tuned=True)
        else:
            nu1, nu2, inner = self._settings(n)
            solver.begin(rho, phi, tol=req.tol, method="mg", prec=self.prec, nu1=nu1, nu2=nu2,
                         max_iter=self.max_iter, inner_cycles=inner)
        return slot

    # ------------------------------------------------------------------ loop
    def run(self, requests, realtime: bool = True, keep_results: bool = False, clock=None):
        """Serve `requests` (arrival_s relative to the start).  With realtime the
        loop follows the wall clock; otherwise every request is available at once."""
        clock = clock or time.perf_counter
        pending = sorted(requests, key=lambda r: (r.arrival_s, r.rid))
        active, results = [], []
        t0 = clock()
        peak_active = 0
        ticks = 0
        while pending or active:
            now = clock() - t0
            # admit in arrival order, skipping sequence members whose previous step
            # has not finished yet
            i = 0
            while i < len(pending) and len(active) < self.max_active:
                req = pending[i]
                if realtime and req.arrival_s > now:
                    break
                if not self._admissible(req):
                    i += 1
                    continue
                slot = self._admit(req, now)
                if slot is None:
                    break                         # wait for memory to be released
                active.append(slot)
                pending.pop(i)
            peak_active = max(peak_active, len(active))
            if not active:
                if pending and realtime:
                    time.sleep(max(0.0, min(pending[0].arrival_s - (clock() - t0), 0.01)))
                elif pending:
                    raise RuntimeError("no request can be admitted within the HBM budget")
                continue
            in_batch = any(sl.bslot >= 0 for sl in active)
            if in_batch:
                self.batch.step(self.k)
            for sl in active:
                if sl.bslot < 0:
                    sl.solver.step(self.k)
            if in_batch:
                bstat, _ = self.batch.poll()
            ticks += 1
            still = []
            for sl in active:
                if sl.bslot >= 0:
                    done = bstat[sl.bslot] != 0
                else:
                    done, _ = sl.solver.poll()
                if not done:
                    still.append(sl)
                    continue
                info = self.batch.remove(sl.bslot) if sl.bslot >= 0 else sl.solver.end()
                t_done = clock() - t0
                r = sl.req
                results.append(Result(r.rid, r.n, r.tol, r.arrival_s, sl.admit_s, t_done,
                                      info.iterations, info.rel_residual, info.status,
                                      r.seq_id, r.seq_step, sl.warm))
                if keep_results:
                    self.final_phi[r.rid] = sl.phi
                self.used -= self.field_bytes(r.n)
                if r.seq_id >= 0:
                    self.warm[r.seq_id] = (sl.phi, r.seq_step)
                    self.used += (r.n + 1) ** 3 * 8
                self.pool.put(r.n, sl.solver)
            active = still
        return results, {"ticks": ticks, "peak_active": peak_active}

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        self.pool.close()


def summarize(results):
    """solves/s over the stream and latency percentiles (seconds)."""
    if not results:
        return {}
    lat = sorted(r.latency_s for r in results)
    p = lambda q: lat[min(len(lat) - 1, max(0, int(round(q * len(lat))) - 1))]
    t_first = min(r.arrival_s for r in results)
    t_last = max(r.done_s for r in results)
    ok = sum(1 for r in results if r.status == 0)
    return {"requests": len(results), "converged": ok,
            "solves_per_s": len(results) / max(t_last - t_first, 1e-9),
            "latency_p50_ms": 1e3 * p(0.50), "latency_p99_ms": 1e3 * p(0.99),
            "latency_mean_ms": 1e3 * statistics.fmean(lat),
            "makespan_s": t_last - t_first}
