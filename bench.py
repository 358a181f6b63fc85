#!/usr/bin/env python
"""Benchmark: 256^3 multigrid solve with the multipole open boundary on GB300.

Workload (one "step" = one whole solve, cold start, to relative residual 1e-10):
256 intervals per axis on the unit cube (255^3 unknowns), FP64, 7-point
Laplacian, V(2,2) cycles with red-black Gauss-Seidel, full weighting, trilinear
prolongation, CG on the 8^3 coarsest level, multipole boundary with l_max = 4;
density = 8 isotropic Gaussians (centres U[0.2,0.8]^3, sigma U[0.02,0.08],
amplitude U[0.5,2], seed 2).  Inputs are synthetic and larger than L2
(rho and phi are 136 MB each in FP64).

value = fine-grid unknown updates per second over the whole solve:
(N-1)^3 x V-cycles / solve time, in GLUPS.  The same solve is also timed in the
mixed FP32 and mixed BF16 refinement modes (FP64 outer residual) for the
FP64-vs-mixed part of the metric.

--impl reference times the FP64 CPU oracle on the host cores instead.
Multi-GPU: independent replicas, one per rank (the solve does not shard).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 256
LMAX = 4
TOL = 1e-10
SEED = 2
WORKLOAD = ("256^3 uniform Cartesian, FP64, 7-point Laplacian, MG V(2,2) red-black GS, full "
            "weighting, trilinear prolongation, CG-solved 8^3 coarsest level, multipole l_max=4, "
            "8 Gaussian blobs seed 2, cold start to rel. residual 1e-10")
FP64_PIPE_PEAK_GOPS = 625.0   # nominal 1.25 TFLOP/s FP64 (FMA = 2 flops) = 625 G FP64 instr/s


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        # raw samples go to BENCH_CLOCKS_DIR (default: the system temp directory);
        # the bench line carries their summary
        base = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(base, f"clocks_{os.getpid()}.csv")
        self.gpu_id = gpu_id

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception as e:  # no nvidia-smi: report nothing rather than guess
            log("clock sampling unavailable:", e)
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ the CPU oracle on the host cores
def _oracle_replica(conn, n):
    """One oracle process: builds the n^3 workload (density, multipole boundary,
    hierarchy), then runs one FP64 V(2,2) cycle per "go" and answers with its
    duration.  numpy runs these stencil loops on one thread, so the host's
    cores are used by running one such process per core."""
    import workloads as W
    from oracle import multigrid as OMG, multipole as OM
    from oracle.grid import cart_grid, hierarchy
    g = cart_grid(n)
    rho = W.gaussian_blobs(n, seed=SEED)
    phi = g.zeros()
    q = OM.moments_cartesian(rho, g, (0.5, 0.5, 0.5), LMAX)
    OM.apply_cartesian_bc(phi, g, q, (0.5, 0.5, 0.5), LMAX, 1.0)
    f = 4 * math.pi * rho
    levels = hierarchy(g)
    conn.send("ready")
    while conn.recv() == "go":
        t0 = time.perf_counter()
        OMG.vcycle(levels, 0, phi, f, 2, 2)
        conn.send(time.perf_counter() - t0)
    conn.close()


def host_replicas(max_procs=None):
    """How many oracle processes the host takes: one per core, at most one per
    2 GB of available memory (a 256^3 oracle V-cycle peaks near 1.2 GB)."""
    cores = os.cpu_count() or 1
    avail = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        avail = None
    n = cores if avail is None else max(1, min(cores, int(avail // 2e9)))
    env = os.environ.get("BENCH_CPU_PROCS")
    if env:
        n = max(1, min(n, int(env)))
    if max_procs is not None:
        n = max(1, min(n, max_procs))
    return n


class OracleReplicas:
    """P spawned oracle processes on the same workload; step() runs one V-cycle
    in each at once and returns the wall time of the slowest."""

    def __init__(self, procs, n=N):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for _ in range(procs):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_replica, args=(b, n), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            if c.recv() != "ready":
                raise RuntimeError("oracle replica failed to start")

    def step(self):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send("go")
        per = [c.recv() for c in self.conns]
        return time.perf_counter() - t0, per

    def close(self):
        for c in self.conns:
            try:
                c.send("stop")
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()


def run_reference(args, rank, world):
    """The FP64 CPU oracle, as it stands, on the host cores: each step is one
    FP64 V(2,2) cycle of the same 256^3 workload in each of P processes (one per
    core, memory permitting).  value = P x (N-1)^3 unknown updates / step time,
    the unit of the GPU arm."""
    if rank != 0:
        return 0
    procs = host_replicas()
    reps = OracleReplicas(procs)
    try:
        for _ in range(args.warmup):
            reps.step()
        walls = []
        for _ in range(args.steps):
            walls.append(reps.step()[0])
    finally:
        reps.close()
    dt = sum(walls)
    value = procs * (N - 1) ** 3 * args.steps / dt / 1e9
    sample = (f"{args.steps} steps, each one FP64 V(2,2) cycle of the 256^3 workload in each of {procs} "
              f"single-threaded numpy processes (oracle/multigrid.vcycle); host has {os.cpu_count()} cores")
    line = {"impl": "reference", "metric": "GLUPS (fine-grid unknown updates/s over the whole solve)",
            "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_n": N},
            "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": procs, "kind": "oracle",
                             "host_cores": os.cpu_count(), "threads_per_process": 1, "sample": sample},
            "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample():
    """The oracle on the host: one FP64 V(2,2) cycle of the same 256^3 workload
    on one core, then one on every core at once (one process per core)."""
    reps = OracleReplicas(1)
    try:
        t1 = reps.step()[0]
    finally:
        reps.close()
    procs = host_replicas()
    if procs > 1:
        reps = OracleReplicas(procs)
        try:
            tp = reps.step()[0]
        finally:
            reps.close()
    else:
        tp = t1
    one = (N - 1) ** 3 / t1 / 1e9
    allc = procs * (N - 1) ** 3 / tp / 1e9
    return {"value": allc, "unit": "GLUPS", "cores": procs, "kind": "oracle",
            "single_core_value": one, "host_cores": os.cpu_count(),
            "sample": f"one FP64 V(2,2) cycle of the 256^3 workload per process, {procs} single-threaded "
                      f"numpy processes at once ({tp:.1f} s); alone on one core {t1:.1f} s"}


# ------------------------------------------------------------------ spherical workload (config 4)
def run_spherical(args, rank, world):
    """256 x 128 x 256 spherical grid (r log-spaced 0.01..1, theta cell-centred,
    phi periodic), rho = r^-2 (1 + 0.1 cos 2 phi)(1 + 0.2 cos^2 theta), multipole
    outer boundary l_max = 6, Neumann inner boundary.  One step = one cold-start
    solve to relative residual --sph-tol (1e-8: the FP64 rounding floor of this
    grid is about 5e-10) or --max-iter iterations: right-Jacobi BiCGSTAB in
    FP64 (--prec fp64) or FP64 refinement around FP32 BiCGSTAB (--prec
    mixed_fp32), or red-black SOR with the local Chebyshev weights (--workload
    sph_sor).  --plain-graphs runs the solves with kernel timing on, whose plain
    graphs (no conditional nodes) a profiler can see into."""
    import torch
    import workloads as W
    import paper_2605_03563_gb300 as P
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    r, th, ph = W.spherical_coords(256, 128, 256, 0.01, 1.0)
    rho = torch.from_numpy(W.spherical_density(r, th, ph)).to(dev)
    phi = torch.zeros_like(rho)
    sor = args.workload == "sph_sor"
    kw = dict(tol=args.sph_tol, max_iter=args.max_iter or 60000)
    if sor:
        kw.update(method="sor", sor_schedule="chebyshev")
    else:
        kw.update(prec=args.prec)
    stream = torch.cuda.current_stream()
    with P.SphericalSolver(r, th, ph, bc="multipole", lmax=6) as s:
        if args.plain_graphs:
            s.profile(True)
        for _ in range(args.warmup):
            s.solve(rho, phi.zero_(), **kw)
        clocks = ClockSampler()
        clocks.start()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        infos = []
        torch.cuda.synchronize()
        ev[0].record(stream)
        for k in range(args.steps):
            infos.append(s.solve(rho, phi.zero_(), **kw))
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        prof = s.profile_read() if args.plain_graphs else {}
    total_ms = ev[0].elapsed_time(ev[args.steps])
    its = sum(i.iterations for i in infos)
    nunk = 256 * 128 * 256
    line = {"metric": "time-to-tolerance (spherical BiCGSTAB / SOR, config 4)",
            "value": total_ms / args.steps, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
            "dtype": "f64" if (sor or args.prec == "fp64") else "f32+f64", "data": "synthetic",
            "config": {"workload": "256x128x256 spherical, l_max 6, " + ("red-black SOR (local Chebyshev)" if sor
                                                                         else "Jacobi-BiCGSTAB " + args.prec),
                       "tol": args.sph_tol, "max_iter": kw["max_iter"], "plain_graphs": bool(args.plain_graphs)},
            "iterations": infos[-1].iterations, "rel_residual": infos[-1].rel_residual,
            "converged": infos[-1].converged, "ms_per_iteration": total_ms / max(its, 1),
            "glups_per_iteration": nunk * its / (total_ms / 1e3) / 1e9,
            "kernels": {k: {"launches": v["launches"], "avg_ms": round(v["avg_ms"], 5)} for k, v in prof.items()},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ serving stream
def run_serving(args, rank, world):
    """2000 Cartesian solve requests (Poisson arrivals, mean 200/s, cubes 32..256,
    1-16 Gaussian blobs, tolerance 1e-6 or 1e-10, 30% warm-started sequence
    steps) served with continuous batching under an HBM budget."""
    import torch
    import workloads as W
    import paper_2605_03563_gb300 as P
    from paper_2605_03563_gb300.serving import PoissonServer, summarize
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    reqs = W.serving_stream(n_requests=args.requests, rate_hz=200.0, seed=5)
    srv = PoissonServer(dev, hbm_budget_bytes=int(args.budget_gb * (1 << 30)), prec=args.prec,
                        cycles_per_step=args.cycles_per_step, max_active=args.max_active,
                        executor=args.executor, max_n=max(r.n for r in reqs))
    # pre-warm: a few handles per size with their loop graphs captured
    warm_reqs = []
    sizes = sorted({r.n for r in reqs})
    for n in sizes:
        for k in range(args.prewarm):
            r = W.ServingRequest(-1 - len(warm_reqs), 0.0, n, 1e-6, W.gaussian_blob_params(99, 2))
            warm_reqs.append(r)
    srv.run(warm_reqs, realtime=False)
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    t0 = time.perf_counter()
    results, stats = srv.run(reqs, realtime=True)
    wall = time.perf_counter() - t0
    # saturated throughput: the same requests all available at once (the
    # arrival rate no longer caps solves/s)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    off_results, off_stats = srv.run(reqs, realtime=False)
    torch.cuda.synchronize()
    off_wall = time.perf_counter() - t1
    clk = clocks.stop()
    srv.close()
    summ = summarize(results)
    by_tol = {}
    for tol in (1e-6, 1e-10):
        sub = [r for r in results if r.tol == tol]
        if sub:
            s2 = summarize(sub)
            by_tol[f"{tol:g}"] = {k: s2[k] for k in ("requests", "latency_p50_ms", "latency_p99_ms")}
    line = {"metric": "solves/s + p50/p99 latency (serving stream)", "value": summ["solves_per_s"],
            "unit": "solves/s", "n_gpus": world, "higher_is_better": True, "dtype": args.prec,
            "data": "synthetic", "scaling": "weak",
            "config": {"workload": "2000 requests, Poisson arrivals 200/s, cubes {32..256}^3, 1-16 "
                                   "Gaussian blobs, tol 1e-6/1e-10, 30% warm-started sequences",
                       "requests": len(reqs), "max_active": args.max_active, "executor": args.executor,
                       "cycles_per_step": args.cycles_per_step, "budget_gb": args.budget_gb},
            "latency_p50_ms": summ["latency_p50_ms"], "latency_p99_ms": summ["latency_p99_ms"],
            "latency_mean_ms": summ["latency_mean_ms"], "by_tol": by_tol,
            "converged": summ["converged"], "makespan_s": summ["makespan_s"], "wall_s": wall,
            "peak_active": stats["peak_active"], "ticks": stats["ticks"],
            "saturated": {"solves_per_s": len(off_results) / off_wall, "wall_s": off_wall,
                          "converged": sum(1 for r in off_results if r.status == 0),
                          "ticks": off_stats["ticks"]},
            "warm_started": sum(1 for r in results if r.warm), "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ the other configurations
def other_configs(dev, reps=3):
    """Time-to-tolerance of the other workloads, each through the public API on
    device-resident inputs (median of `reps` solves after one warm-up):
      config 1: 32^3 uniform sphere, analytic Dirichlet boundary, SOR (omega 1.8, the Chebyshev
                weights of Eq. omega_n and omega_opt of Eq. 3), CG and multicolour-Gauss-Seidel-
                preconditioned CG to 1e-10;
      config 3: 512^3 lognormal density, 13-point, multipole l_max = 8, MG to 1e-10 in FP64 and
                in the FP32-smoothing / BF16-finest refinement mode;
      config 4: 256 x 128 x 256 spherical grid, multipole l_max = 6, Jacobi-BiCGSTAB to 1e-8 (the
                exact solution rounded to FP64 has a residual near 5e-10 on this grid) in FP64 and
                as FP64 refinement around FP32-vector inner solves, and red-black SOR with per-node
                Chebyshev weights from the local rJ of Eq. local_rjac."""
    import torch
    import workloads as W
    import paper_2605_03563_gb300 as P
    out = {}

    def timed(fn, reps_):
        fn()
        ts, info = [], None
        for _ in range(reps_):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            info = fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts), info

    # config 1
    rho_np, phi0_np, _ = W.uniform_sphere(32)
    rho1 = torch.from_numpy(rho_np).to(dev)
    phi0 = torch.from_numpy(phi0_np).to(dev)
    c1 = {}
    with P.CartesianSolver(32) as s:
        for name, method, omega, sched in (("sor", "sor", 1.8, "fixed"), ("sor_chebyshev", "sor", 1.0, "chebyshev"),
                                           ("sor_optimal", "sor", 1.0, "optimal"), ("cg", "cg", 1.0, "fixed"),
                                           ("pcg", "pcg", 1.0, "fixed")):
            phi = phi0.clone()

            def run():
                phi.copy_(phi0)
                return s.solve(rho1, phi, tol=1e-10, method=method, omega=omega, max_iter=20000,
                               sor_schedule=sched)
            ms, info = timed(run, 10)
            c1[name] = {"time_to_1e-10_ms": ms, "iterations": info.iterations,
                          "rel_residual": info.rel_residual, "converged": info.converged,
                          "glups_per_step": 31 ** 3 * info.iterations / (ms / 1e3) / 1e9}
    out["config1_32_sphere_sor_cg"] = c1

    # config 3
    n3 = 512
    rho3 = W.lognormal_field_device(n3, dev, order=4, seed=3)
    c3 = {}
    with P.CartesianSolver(n3, 4, bc="multipole", lmax=8) as s:
        ref = None
        for prec, inner in (("fp64", 1), ("mixed_bf16", 2), ("mixed_fp32", 2)):
            phi = torch.zeros_like(rho3)

            def run():
                phi.zero_()
                return s.solve(rho3, phi, tol=1e-10, method="mg", prec=prec, max_iter=60,
                               inner_cycles=inner)
            ms, info = timed(run, reps)
            rec = {"time_to_1e-10_ms": ms, "iterations": info.iterations, "converged": info.converged,
                   "rel_residual": info.rel_residual, "inner_vcycles": info.inner_cycles,
                   "t_mp_ms": info.t_mp_ms}
            if prec == "fp64":
                ref = phi.clone()
                rec["glups"] = (n3 - 1) ** 3 * info.iterations / (ms / 1e3) / 1e9
            else:
                rec["max_rel_diff_vs_fp64_gpu"] = float((phi - ref).abs().max() / ref.abs().max())
                rec["speedup_vs_fp64"] = c3["fp64"]["time_to_1e-10_ms"] / ms
            c3[prec] = rec
        del ref
    del rho3
    out["config3_512_lognormal_13pt"] = c3

    # config 4
    r, th, ph_ = W.spherical_coords(256, 128, 256, 0.01, 1.0)
    rho4 = torch.from_numpy(W.spherical_density(r, th, ph_)).to(dev)
    with P.SphericalSolver(r, th, ph_, bc="multipole", lmax=6) as s:
        phi = torch.zeros_like(rho4)

        def run():
            phi.zero_()
            return s.solve(rho4, phi, tol=1e-8, max_iter=40000)
        ms, info = timed(run, 1)
        nunk = 256 * 128 * 256
        out["config4_spherical_bicgstab_fp64"] = {
            "time_to_1e-8_ms": ms, "iterations": info.iterations, "converged": info.converged,
            "rel_residual": info.rel_residual, "t_mp_ms": info.t_mp_ms,
            "ms_per_iteration": ms / max(info.iterations, 1),
            "glups_per_iteration": nunk * info.iterations / (ms / 1e3) / 1e9}
        ref4 = phi.clone()

        def run_mixed():
            phi.zero_()
            return s.solve(rho4, phi, tol=1e-8, max_iter=80000, prec="mixed_fp32")
        ms, info = timed(run_mixed, 1)
        out["config4_spherical_bicgstab_mixed_fp32"] = {
            "time_to_1e-8_ms": ms, "iterations": info.iterations, "converged": info.converged,
            "rel_residual": info.rel_residual, "inner_solves": info.inner_cycles,
            "ms_per_iteration": ms / max(info.iterations, 1),
            "max_rel_diff_vs_fp64_gpu": float((phi - ref4).abs().max() / ref4.abs().max()),
            "speedup_vs_fp64": out["config4_spherical_bicgstab_fp64"]["time_to_1e-8_ms"] / ms}
        del ref4

        def run_sor():
            phi.zero_()
            return s.solve(rho4, phi, tol=1e-8, max_iter=40000, method="sor", sor_schedule="chebyshev")
        ms, info = timed(run_sor, 1)
        out["config4_spherical_sor_chebyshev_fp64"] = {
            "time_to_1e-8_ms": ms, "iterations": info.iterations, "converged": info.converged,
            "rel_residual": info.rel_residual, "ms_per_step": ms / max(info.iterations, 1),
            "glups_per_step": nunk * info.iterations / (ms / 1e3) / 1e9}
    return out


# ------------------------------------------------------------------ compact-stencil MG (Table 4's method)
def compact_mg(dev, sizes=(256, 512), nus=(1, 2, 3), reps=2, precs=("fp64", "mixed_fp32")):
    """The paper's sixth-order multigrid (Sec. 2.1.3: compact radius-one stencil,
    SPAI smoothing with Table 1's coefficients, Galerkin coarse operators) on the
    two-sphere problem of Sec. 3.1 (two (1 - w^2)^2 spheres, radii 0.08, masses 1
    and 2, centred at z = 0.4 and -0.2 on [-1, 1]^3), multipole boundary l_max 4,
    cold start to residual reduction 1e-6, as in Table 4: V-cycles, t_mp, t_iter,
    t_s (per V-cycle) and s_s = (N-1)^3 / t_s; in FP64 and as FP64 refinement
    around FP32 inner V-cycles (inner V-cycles per refinement step tuned among
    1-4, every trial reported; t_s per inner V-cycle)."""
    import torch
    import workloads as W
    import paper_2605_03563_gb300 as P
    out = {}
    for n in sizes:
        rho = torch.from_numpy(W.smooth_sphere_density(n, 2, [(0.0, 0.0, 0.4), (0.0, 0.0, -0.2)],
                                                       [0.08, 0.08], [1.0, 2.0])).to(dev)
        with P.CartesianSolver(n, 2, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), bc="multipole", lmax=4) as s:
            for prec, nu in [(p_, nu_) for p_ in precs for nu_ in nus]:
                phi = torch.zeros_like(rho)

                def run(inner):
                    phi.zero_()
                    return s.solve(rho, phi, tol=1e-6, method="mg", prec=prec, nu1=nu, nu2=nu, max_iter=40,
                                   inner_cycles=inner, compact_order=6)

                def timed(inner):
                    run(inner)
                    torch.cuda.synchronize()
                    ts, info = [], None
                    for _ in range(reps):
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record()
                        info = run(inner)
                        b.record()
                        torch.cuda.synchronize()
                        ts.append(a.elapsed_time(b))
                    return min(ts), info
                # FP32 refinement: inner V-cycles per refinement step tuned among 1-4
                cands = (1,) if prec == "fp64" else (1, 2, 3, 4)
                trials = {c: timed(c) for c in cands}
                best = min((c for c in cands if trials[c][1].converged), key=lambda c: trials[c][0])
                ms, info = trials[best]
                t_iter = ms - info.t_mp_ms
                cyc = max(info.iterations * (best if prec != "fp64" else 1), 1)
                out[f"n{n - 1}_nu{nu}_{prec}"] = {
                    "v_cycles": cyc, "steps": info.iterations, "converged": info.converged,
                    "rel_residual": info.rel_residual, "time_to_1e-6_ms": ms, "t_mp_ms": info.t_mp_ms,
                    "t_iter_ms": t_iter, "t_s_ms": t_iter / cyc, "rho_conv": info.rho_conv,
                    "s_s_gzups": (n - 1) ** 3 / (t_iter / cyc / 1e3) / 1e9}
                if prec != "fp64":
                    out[f"n{n - 1}_nu{nu}_{prec}"]["inner_cycles"] = best
                    out[f"n{n - 1}_nu{nu}_{prec}"]["trials"] = {
                        c: {"time_to_1e-6_ms": trials[c][0], "steps": trials[c][1].iterations,
                            "converged": trials[c][1].converged} for c in cands}
                if nu == max(nus):
                    # per-kernel CUDA-event times of one more solve (plain graphs with
                    # event nodes around the hot kernels)
                    s.profile(True)
                    s.profile_read()
                    run(best)
                    torch.cuda.synchronize()
                    pr = s.profile_read()
                    s.profile(False)
                    out[f"n{n - 1}_nu{nu}_{prec}"]["kernels"] = {
                        k: {"launches": v["launches"], "avg_ms": round(v["avg_ms"], 5),
                            "total_ms": round(v["total_ms"], 4),
                            "GB/s": round(v["bytes_per_launch"] / (v["avg_ms"] / 1e3) / 1e9, 1)
                            if v["avg_ms"] > 0 else None}
                        for k, v in sorted(pr.items(), key=lambda kv: -kv[1]["total_ms"])}
        del rho
    return out


# ------------------------------------------------------------------ batched throughput
def batched_throughput(dev, per_size=8, sizes=(32, 64, 96, 128, 192, 256), reps=2):
    """Solves/s to relative residual 1e-10 on a fixed set of grids of the serving
    mix (per_size Gaussian-mixture densities of every size): the plain FP64 path
    (one poisson_solve after another) against the batched executor (every grid
    in one batch, one graph launch per step) in FP64 and with FP32 refinement.
    Potentials of the batched mixed mode are compared with the FP64 ones."""
    import torch
    import workloads as W
    import paper_2605_03563_gb300 as P
    grids = []
    for n in sizes:
        for k in range(per_size):
            rho = W.gaussian_blobs_device(n, W.gaussian_blob_params(1000 + 17 * n + k, 1 + (k % 16)), dev)
            grids.append((n, rho))
    solvers = [P.CartesianSolver(n, bc="multipole", lmax=LMAX) for n, _ in grids]
    phis64 = [torch.zeros_like(r) for _, r in grids]
    out = {"grids": len(grids), "sizes": list(sizes), "per_size": per_size, "tol": TOL}
    try:
        def plain():
            for s, (n, rho), phi in zip(solvers, grids, phis64):
                phi.zero_()
                s.solve(rho, phi, tol=TOL, method="mg", max_iter=100)
        plain()
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            t0 = time.perf_counter()
            plain()
            torch.cuda.synchronize()
            t.append(time.perf_counter() - t0)
        out["plain_fp64_solves_per_s"] = len(grids) / min(t)

        def batched(prec, inner, nu=(2, 2)):
            with P.Batch(len(grids), max(sizes), prec=prec, inner_cycles=inner, nu1=nu[0], nu2=nu[1]) as b:
                phis = [torch.zeros_like(r) for _, r in grids]

                def run():
                    for p_ in phis:
                        p_.zero_()
                    slots = [b.add(s, rho, p_, tol=TOL, max_iter=100)
                             for s, (_, rho), p_ in zip(solvers, grids, phis)]
                    while True:
                        st, _ = b.poll()
                        if all(st[sl] != 0 for sl in slots):
                            break
                        b.step(2)
                    infos = [b.remove(sl) for sl in slots]
                    torch.cuda.synchronize()
                    return infos
                run()
                ts = []
                for _ in range(reps):
                    t0 = time.perf_counter()
                    infos = run()
                    ts.append(time.perf_counter() - t0)
                assert all(i.converged for i in infos)
                err = max(float((p_ - q).abs().max() / q.abs().max()) for p_, q in zip(phis, phis64))
                return len(grids) / min(ts), err
        def hybrid(prec, inner, batch_max_n=96):
            # grids up to batch_max_n share the batched executor's graph launches;
            # larger ones run their own loop graphs (tile kernels on their finest
            # levels) on their handles' streams, concurrently with the batch
            small = [i for i, (n, _) in enumerate(grids) if n <= batch_max_n]
            large = [i for i, (n, _) in enumerate(grids) if n > batch_max_n]
            phis = [torch.zeros_like(r) for _, r in grids]
            with P.Batch(max(1, len(small)), batch_max_n, prec=prec, inner_cycles=inner) as b:
                def run():
                    for p_ in phis:
                        p_.zero_()
                    for i in large:
                        solvers[i].begin(grids[i][1], phis[i], tol=TOL, method="mg", prec=prec,
                                         max_iter=100, inner_cycles=inner)
                        solvers[i].step(100)        # the loop graph stops at convergence
                    slots = [b.add(solvers[i], grids[i][1], phis[i], tol=TOL, max_iter=100) for i in small]
                    while slots:
                        st, _ = b.poll()
                        if all(st[sl] != 0 for sl in slots):
                            break
                        b.step(2)
                    infos = [b.remove(sl) for sl in slots] + [solvers[i].end() for i in large]
                    torch.cuda.synchronize()
                    return infos
                run()
                ts = []
                for _ in range(reps):
                    t0 = time.perf_counter()
                    infos = run()
                    ts.append(time.perf_counter() - t0)
            assert all(i.converged for i in infos)
            err = max(float((p_ - q).abs().max() / q.abs().max()) for p_, q in zip(phis, phis64))
            return len(grids) / min(ts), err
        out["batched_fp64_solves_per_s"], e64 = batched("fp64", 1)
        # the batch's cycle shape and inner V-cycles per refinement step, tuned
        trials = {}
        for nu in ((2, 2), (2, 1), (1, 1)):
            for inner in (1, 2, 3):
                trials[f"V({nu[0]},{nu[1]}) inner {inner}"] = batched("mixed_fp32", inner, nu)
        best = max(trials, key=lambda k: trials[k][0])
        out["batched_mixed_fp32_solves_per_s"], emx = trials[best]
        out["batched_mixed_fp32_setting"] = best
        out["batched_mixed_fp32_trials"] = {k: v[0] for k, v in trials.items()}
        out["hybrid_fp64_solves_per_s"], eh64 = hybrid("fp64", 1)
        out["hybrid_mixed_fp32_solves_per_s"], ehmx = hybrid("mixed_fp32", 2)
        out["batched_fp64_max_rel_diff_vs_plain"] = e64
        out["batched_mixed_max_rel_diff_vs_plain_fp64"] = emx
        out["hybrid_fp64_max_rel_diff_vs_plain"] = eh64
        out["hybrid_mixed_max_rel_diff_vs_plain_fp64"] = ehmx
        out["mixed_batched_vs_plain_fp64"] = out["batched_mixed_fp32_solves_per_s"] / out["plain_fp64_solves_per_s"]
        out["mixed_hybrid_vs_plain_fp64"] = out["hybrid_mixed_fp32_solves_per_s"] / out["plain_fp64_solves_per_s"]
    finally:
        for s in solvers:
            s.close()
    return out


# ------------------------------------------------------------------ FP64 pipe peak, bench line
def fp64_peak(dev):
    """Measured FP64 instruction rate of this GPU (G instructions/s, warp lanes
    counted one by one): the library's probe kernel, 8 blocks per SM, timed
    with CUDA events (best of 3 after one warm-up launch), for fused
    multiply-adds and for adds."""
    import torch
    from paper_2605_03563_gb300 import ops
    blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 8
    out = torch.empty(blocks, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    for kind, name in ((0, "dfma"), (1, "dadd")):
        times, n = [], 0.0
        for it in range(4):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            n = ops.probe_fp64(kind, blocks, 2048, out, stream)
            b.record(stream)
            torch.cuda.synchronize()
            if it > 0:
                times.append(a.elapsed_time(b))
        res[name] = n / (min(times) / 1e3) / 1e9
    return res


HEADLINE_MAX_BYTES = 3072


def _r(x, nd=4):
    if isinstance(x, float):
        return float(f"{x:.{nd}g}")
    return x


def _clip(x, n=240):
    return x[:n] if isinstance(x, str) else x


def write_details(full):
    """Everything the run measured, as one JSON file in BENCH_DETAILS_DIR (default:
    the system temp directory); returns its path."""
    base = os.environ.get("BENCH_DETAILS_DIR") or tempfile.gettempdir()
    try:
        os.makedirs(base, exist_ok=True)
        path = os.path.join(base, f"bench_details_{os.getpid()}.json")
        with open(path, "w") as f:
            json.dump(full, f, indent=1)
        return path
    except OSError:
        return None


def headline(full, details_path=None):
    """The one line rank 0 prints: the keys a reader of the run needs (metric,
    value, timing, config, roofline, CPU baseline, end-to-end, clocks, and the
    FP64-vs-mixed figures), a few KB at most; everything else stays in the
    details file."""
    keep = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "gpu_launches")
    line = {k: full.get(k) for k in keep}
    cfg = full.get("config") or {}
    line["config"] = {k: cfg[k] for k in ("workload", "n_intervals", "l_max", "tol", "v_cycles_per_solve",
                                           "l2", "parallelism") if k in cfg}
    if isinstance(line["config"].get("workload"), str):
        line["config"]["workload"] = line["config"]["workload"][:400]
    t = full.get("time_to_1e-10_ms") or {}
    line["time_to_1e-10_ms"] = {k: _r(v) for k, v in t.items()}
    mixed = {}
    for prec, m in (full.get("mixed") or {}).items():
        mixed[prec] = {k: _r(m.get(k)) for k in ("time_to_1e-10_ms", "speedup_vs_fp64", "inner_cycles",
                                                  "ir_steps", "max_rel_diff_vs_fp64_gpu", "converged")}
    line["mixed"] = mixed
    roof = full.get("roofline") or {}
    line["roofline"] = {k: _r(v) for k, v in roof.items()
                        if k in ("bound", "kernel", "achieved", "peak", "unit", "frac", "traffic",
                                 "hbm_achieved_gbs", "hbm_peak_gbs", "hbm_frac", "hbm_frac_3S",
                                 "algorithmic_bytes_per_launch", "algorithmic_bytes_3S", "avg_launch_ms",
                                 "fp64_dadd_peak", "peak_source")}
    cpu = full.get("cpu_baseline")
    line["cpu_baseline"] = None if cpu is None else {k: _clip(_r(v)) for k, v in cpu.items()}
    e2e = full.get("e2e") or {}
    line["e2e"] = {k: _clip(_r(v)) for k, v in e2e.items()}
    clk = full.get("clocks")
    line["clocks"] = clk
    b = full.get("batched") or {}
    if b:
        line["batched"] = {k: _r(b[k]) for k in ("plain_fp64_solves_per_s", "batched_mixed_fp32_solves_per_s",
                                                  "hybrid_mixed_fp32_solves_per_s", "mixed_batched_vs_plain_fp64",
                                                  "mixed_hybrid_vs_plain_fp64") if k in b}
    line["details"] = details_path if details_path is None or len(details_path) < 200 else None
    text = json.dumps(line)
    for drop in ("batched", "mixed", "details"):
        if len(text) <= HEADLINE_MAX_BYTES:
            break
        line.pop(drop, None)
        text = json.dumps(line)
    return line


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="mg256", choices=["mg256", "serving", "sph", "sph_sor"])
    ap.add_argument("--sph-tol", type=float, default=1e-8, help="spherical workloads: relative residual")
    ap.add_argument("--max-iter", type=int, default=0, help="spherical workloads: iteration cap (0 = 60000)")
    ap.add_argument("--plain-graphs", action="store_true",
                    help="spherical workloads: solve with kernel timing on (plain graphs a profiler can see into)")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "mixed_fp32", "mixed_bf16"])
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--max-active", type=int, default=64)
    ap.add_argument("--cycles-per-step", type=int, default=2)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--prewarm", type=int, default=4)
    ap.add_argument("--executor", default="hybrid", choices=["batch", "streams", "hybrid"],
                    help="serving: batched executor (one graph launch per tick for all solves), "
                         "per-request graphs, or the batch for grids up to 96^3 and graphs above")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the timings of the other configurations, the batched executor and "
                         "the compact multigrid (same as --configs none)")
    ap.add_argument("--configs", default="other,batched,compact",
                    help="comma-separated subset of other (configurations 1, 3, 4), batched "
                         "(batched executor throughput) and compact (sixth-order multigrid on the "
                         "two-sphere problem), or none")
    ap.add_argument("--compact-sizes", default="256,512",
                    help="grid sizes (intervals) of the compact multigrid timings")
    ap.add_argument("--tile-min-n", type=int, default=0,
                    help="levels with at least this many intervals use the TMA tile kernels "
                         "(0 = library default, -1 = never)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "serving":
        return run_serving(args, rank, world)
    if args.workload in ("sph", "sph_sor"):
        return run_spherical(args, rank, world)

    import numpy as np
    import torch
    import workloads as W
    import paper_2605_03563_gb300 as P

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    rho_h = torch.from_numpy(W.gaussian_blobs(N, seed=SEED)).pin_memory()
    rho = rho_h.to(dev)
    phi = torch.zeros_like(rho)
    stream = torch.cuda.current_stream()
    solver = P.CartesianSolver(N, bc="multipole", lmax=LMAX)

    def one(prec="fp64", out=None):
        out = phi if out is None else out
        out.zero_()
        return solver.solve(rho, out, tol=TOL, method="mg", prec=prec, max_iter=100,
                            tile_min_n=args.tile_min_n)

    for _ in range(args.warmup):
        info = one()
    assert info.converged, info

    # ---- timed FP64 region
    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    clocks = ClockSampler(gpu_id)
    infos, ev = [], [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev[0].record(stream)
    for k in range(args.steps):
        infos.append(one())
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[args.steps])
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    cycles = [i.iterations for i in infos]
    assert all(i.converged for i in infos), infos[-1]
    unknowns = (N - 1) ** 3
    value = world * unknowns * sum(cycles) / (total_ms / 1e3) / 1e9
    launches = sum(i.kernel_launches for i in infos)
    phi64 = phi.clone()

    # ---- per-kernel durations: the same solves again with CUDA events recorded
    # on the solve stream around each hot kernel (event records cannot live
    # inside the captured loop graphs, so this region launches kernels directly)
    solver.profile(True)
    prof_steps = max(3, args.steps // 2)
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pa.record(stream)
    for _ in range(prof_steps):
        one()
    pb.record(stream)
    torch.cuda.synchronize()
    prof_region_ms = pa.elapsed_time(pb) / prof_steps
    prof = solver.profile_read()
    solver.profile(False)

    # ---- end to end through the public API with host buffers: every step copies
    # its input (rho) from pinned host memory and reads its potential back (a
    # cold start: the initial guess is zeroed on the device, not copied); two
    # device buffer sets let the copy of step k + 1 (and the read-back of step
    # k) run on a copy stream while step k solves
    phi_out_h = [torch.empty_like(rho_h).pin_memory() for _ in range(2)]
    rho_d = [torch.empty_like(rho) for _ in range(2)]
    phi_d = [torch.empty_like(rho) for _ in range(2)]
    ready = [torch.cuda.Event() for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    solve_stream = torch.cuda.Stream(device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_cycles = 0

    def h2d(slot):
        with torch.cuda.stream(copy_stream):
            rho_d[slot].copy_(rho_h, non_blocking=True)
            phi_d[slot].zero_()
            ready[slot].record(copy_stream)

    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    copy_stream.wait_stream(stream)
    solve_stream.wait_stream(stream)
    h2d(0)
    for k in range(args.steps):
        slot = k % 2
        if k + 1 < args.steps:
            h2d(1 - slot)   # the other set's last solve has returned; its read-back precedes on the copy stream
        solve_stream.wait_event(ready[slot])
        inf = solver.solve(rho_d[slot], phi_d[slot], tol=TOL, method="mg", max_iter=100,
                           tile_min_n=args.tile_min_n, stream=solve_stream)
        e2e_cycles += inf.iterations
        copy_stream.wait_stream(solve_stream)
        with torch.cuda.stream(copy_stream):
            phi_out_h[slot].copy_(phi_d[slot], non_blocking=True)
    stream.wait_stream(copy_stream)
    stream.wait_stream(solve_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_value = world * unknowns * e2e_cycles / (e2e_ms / 1e3) / 1e9
    nbytes = rho_h.numel() * 8

    # ---- mixed precision variants (same workload, same tolerance): the number of
    # inner V-cycles per refinement step is autotuned (1, 2 or 3), every trial is
    # reported, and the best one is profiled for its kernels' HBM rooflines
    peaks, peak_src = measured_peaks()

    def kernel_table(pr):
        tot = sum(x["total_ms"] for x in pr.values()) or 1.0
        out = {}
        for k, v in pr.items():
            sec = v["avg_ms"] / 1e3
            out[k] = {"launches": v["launches"], "avg_ms": round(v["avg_ms"], 5),
                      "share_of_profiled": round(v["total_ms"] / tot, 4),
                      "GB/s": round(v["bytes_per_launch"] / sec / 1e9, 1) if sec > 0 else None,
                      "hbm_frac": round(v["bytes_per_launch"] / sec / 1e9 / peaks["hbm_gbs"], 3) if sec > 0 else None,
                      "Gop/s": round(v["ops_per_launch"] / sec / 1e9, 1) if sec > 0 else None,
                      "fp64": v["fp64"]}
        return out

    mixed = {}
    if not args.no_mixed:
        reps = max(3, args.steps // 2)
        for prec in ("mixed_fp32", "mixed_bf16"):
            out = torch.zeros_like(rho)
            trials = {}
            for inner in (1, 2, 3):
                for _ in range(2):
                    out.zero_()
                    solver.solve(rho, out, tol=TOL, method="mg", prec=prec, inner_cycles=inner,
                                 tile_min_n=args.tile_min_n)
                times = []
                for _ in range(reps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    out.zero_()
                    a.record(stream)
                    inf = solver.solve(rho, out, tol=TOL, method="mg", prec=prec, inner_cycles=inner,
                                 tile_min_n=args.tile_min_n)
                    b.record(stream)
                    torch.cuda.synchronize()
                    times.append(a.elapsed_time(b))
                trials[inner] = {"time_to_1e-10_ms": statistics.median(times), "ir_steps": inf.iterations,
                                 "inner_vcycles": inf.inner_cycles, "converged": inf.converged,
                                 "rel_residual": inf.rel_residual}
            best = min((t for t in trials if trials[t]["converged"]), key=lambda t: trials[t]["time_to_1e-10_ms"])
            out.zero_()
            inf = solver.solve(rho, out, tol=TOL, method="mg", prec=prec, inner_cycles=best,
                         tile_min_n=args.tile_min_n)
            err = float((out - phi64).abs().max() / phi64.abs().max())
            solver.profile(True)
            for _ in range(2):
                out.zero_()
                solver.solve(rho, out, tol=TOL, method="mg", prec=prec, inner_cycles=best,
                         tile_min_n=args.tile_min_n)
            pr = solver.profile_read()
            solver.profile(False)
            t_best = trials[best]["time_to_1e-10_ms"]
            mixed[prec] = {"inner_cycles": best, "time_to_1e-10_ms": t_best,
                           "ir_steps": trials[best]["ir_steps"], "inner_vcycles": trials[best]["inner_vcycles"],
                           "rel_residual": inf.rel_residual, "max_rel_diff_vs_fp64_gpu": err,
                           "speedup_vs_fp64": statistics.median(step_ms) / t_best,
                           "solves_per_s": 1e3 / t_best, "converged": inf.converged,
                           "trials": trials, "kernels": kernel_table(pr)}

    # ---- roofline of the dominant kernel
    dom_name, dom = max(prof.items(), key=lambda kv: kv[1]["total_ms"])
    traffic = None   # DRAM bytes per launch from the committed ncu capture of that kernel
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            traffic = json.load(f).get(dom_name, {}).get("dram_bytes_per_launch")
    except Exception:
        traffic = None
    avg_s = dom["avg_ms"] / 1e3
    gbs = dom["bytes_per_launch"] / avg_s / 1e9
    gops = dom["ops_per_launch"] / avg_s / 1e9
    fp64_rate = fp64_peak(dev)
    if dom["fp64"]:
        roof = {"bound": "alu", "kernel": dom_name, "achieved": gops, "peak": fp64_rate["dfma"],
                "unit": "G FP64 instr/s (FMA = 1)", "frac": gops / fp64_rate["dfma"],
                "traffic": traffic, "hbm_achieved_gbs": gbs, "hbm_peak_gbs": peaks["hbm_gbs"],
                "hbm_frac": gbs / peaks["hbm_gbs"],
                "algorithmic_bytes_per_launch": dom["bytes_per_launch"],
                "ops_per_launch": dom["ops_per_launch"], "avg_launch_ms": dom["avg_ms"],
                "fp64_dadd_peak": fp64_rate["dadd"],
                "peak_source": "measured in this run: ps_probe_fp64 (DFMA chains, CUDA events); hbm " + peak_src}
        if dom_name == "sweep_colour_finest":
            # the minimal count: 3S per unknown per full red-black sweep (phi and
            # fs read once, phi written once), i.e. 12 B per unknown per colour
            # pass (FP64)
            sb = unknowns * 3 * 8 / 2
            roof["hbm_frac_3S"] = sb / avg_s / 1e9 / peaks["hbm_gbs"]
            roof["algorithmic_bytes_3S"] = sb
    else:
        roof = {"bound": "hbm", "kernel": dom_name, "achieved": gbs, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"], "traffic": traffic,
                "algorithmic_bytes_per_launch": dom["bytes_per_launch"], "avg_launch_ms": dom["avg_ms"],
                "peak_source": peak_src}
    kernels = kernel_table(prof)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_sample()
    configs = None
    batched = None
    compact = None
    extra = set() if args.no_configs else {c.strip() for c in args.configs.split(",") if c.strip()}
    unknown = extra - {"other", "batched", "compact", "none"}
    if unknown:
        raise SystemExit(f"--configs: unknown entries {sorted(unknown)}")
    if rank == 0:
        if "other" in extra:
            configs = other_configs(dev)
        if "batched" in extra:
            batched = batched_throughput(dev)
        if "compact" in extra:
            compact = compact_mg(dev, sizes=tuple(int(v) for v in args.compact_sizes.split(",")))

    solver.close()
    if rank == 0:
        sorted_ms = sorted(step_ms)
        p99 = sorted_ms[min(len(sorted_ms) - 1, int(math.ceil(0.99 * len(sorted_ms))) - 1)]
        full = {
            "metric": "GLUPS (fine-grid unknown updates/s over the whole solve) + time-to-1e-10",
            "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_intervals": N, "unknowns": unknowns, "l_max": LMAX,
                       "tol": TOL, "v_cycles_per_solve": cycles[0], "tile_min_n": args.tile_min_n,
                       "l2": "inputs larger than L2 (rho, phi, scaled RHS: 136 MB each)",
                       "parallelism": f"replicas x{world}"},
            "time_to_1e-10_ms": {"p50": statistics.median(step_ms), "p99": p99,
                                 "mean": total_ms / args.steps},
            "s_t_glups": unknowns / (statistics.median(step_ms) / 1e3) / 1e9,
            "t_mp_ms": infos[-1].t_mp_ms, "rel_residual": infos[-1].rel_residual,
            "rho_conv": infos[-1].rho_conv,
            "mixed": mixed,
            "other_configs": configs,
            "batched": batched,
            "compact_mg_table4": compact,
            "roofline": roof,
            "fp64_pipe_gops": fp64_rate,
            "kernels": kernels,
            "profiled_region_ms_per_step": prof_region_ms,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "GLUPS", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_ms / args.steps,
                    "copies": "pinned host buffers: rho in, the potential out (cold start: the initial "
                              "guess is zeroed on the device); step k+1's copy and step k's read-back "
                              "overlap step k's solve on a copy stream (two device buffer sets)"},
            "gpu_launches": launches,
            "clocks": clk,
        }
        path = write_details(full)
        line = headline(full, path)
        log("bench details:", json.dumps(full))
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
