"""The line bench.py prints last stays small and parseable whatever the run
measured (the full record goes to a details file)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _kernel_table(k):
    return {f"kernel_{i}": {"launches": 100 + i, "avg_ms": 0.123456789, "share_of_profiled": 0.01,
                            "GB/s": 1234.5, "hbm_frac": 0.2, "Gop/s": 555.5, "fp64": True} for i in range(k)}


def _full_record():
    trials = {i: {"time_to_1e-10_ms": 5.123456, "ir_steps": 10, "inner_vcycles": 10, "converged": True,
                  "rel_residual": 9.1e-11} for i in (1, 2, 3)}
    mixed = {p: {"inner_cycles": 2, "time_to_1e-10_ms": 5.77123, "ir_steps": 5, "inner_vcycles": 10,
                 "rel_residual": 8.8e-11, "max_rel_diff_vs_fp64_gpu": 8.9e-11, "speedup_vs_fp64": 2.7512345,
                 "solves_per_s": 173.3, "converged": True, "trials": trials, "kernels": _kernel_table(15)}
             for p in ("mixed_fp32", "mixed_bf16")}
    return {
        "metric": "GLUPS (fine-grid unknown updates/s over the whole solve) + time-to-1e-10",
        "value": 9.391234567, "unit": "GLUPS", "n_gpus": 1, "steps": 20, "warmup": 5,
        "ms_per_step": 15.891234, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "x" * 260, "n_intervals": 256, "unknowns": 255 ** 3, "l_max": 4, "tol": 1e-10,
                   "v_cycles_per_solve": 9, "tile_min_n": 0, "l2": "inputs larger than L2 (136 MB each)",
                   "parallelism": "replicas x1"},
        "time_to_1e-10_ms": {"p50": 15.89, "p99": 16.2, "mean": 15.9},
        "mixed": mixed,
        "other_configs": {"config1": {f"k{i}": {"time_ms": 1.0} for i in range(50)}},
        "batched": {"plain_fp64_solves_per_s": 173.6, "batched_mixed_fp32_solves_per_s": 341.9,
                    "hybrid_mixed_fp32_solves_per_s": 636.9, "mixed_batched_vs_plain_fp64": 1.97,
                    "mixed_hybrid_vs_plain_fp64": 3.67, "grids": 48},
        "compact_mg_table4": {f"n{i}": {"kernels": _kernel_table(12)} for i in range(12)},
        "roofline": {"bound": "alu", "kernel": "sweep_colour_finest", "achieved": 467.1, "peak": 598.2,
                     "unit": "G FP64 instr/s (FMA = 1)", "frac": 0.78, "traffic": 360800000.0,
                     "hbm_achieved_gbs": 2480.0, "hbm_peak_gbs": 6681.5, "hbm_frac": 0.37, "hbm_frac_3S": 0.28,
                     "algorithmic_bytes_per_launch": 265300000.0, "algorithmic_bytes_3S": 199000000.0,
                     "ops_per_launch": 49700000.0, "avg_launch_ms": 0.107, "fp64_dadd_peak": 504.0,
                     "peak_source": "measured in this run: ps_probe_fp64 (DFMA chains, CUDA events); hbm measured"},
        "fp64_pipe_gops": {"dfma": 598.2, "dadd": 504.0},
        "kernels": _kernel_table(15),
        "cpu_baseline": {"value": 0.05, "unit": "GLUPS", "cores": 16, "kind": "oracle", "single_core_value": 0.004,
                         "host_cores": 16, "sample": "s" * 160},
        "e2e": {"value": 8.9, "unit": "GLUPS", "h2d_bytes_per_step": 2 * 136 * 10 ** 6,
                "d2h_bytes_per_step": 136 * 10 ** 6, "ms_per_step": 16.75, "copies": "c" * 150},
        "gpu_launches": 123456,
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 300},
    }


def test_headline_is_small_and_carries_the_driver_keys():
    import bench
    full = _full_record()
    line = bench.headline(full, "/tmp/bench_details_1.json")
    text = json.dumps(line)
    assert len(text) <= bench.HEADLINE_MAX_BYTES, len(text)
    back = json.loads(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "dtype", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in back, k
    assert back["value"] == full["value"]
    assert back["steps"] == 20 and back["warmup"] == 5
    assert back["config"]["workload"] == full["config"]["workload"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in back["roofline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step", "copies"):
        assert k in back["e2e"], k
    assert back["e2e"]["h2d_bytes_per_step"] > 0 and back["e2e"]["d2h_bytes_per_step"] > 0
    assert back["cpu_baseline"]["cores"] == 16
    assert back["mixed"]["mixed_fp32"]["speedup_vs_fp64"] > 1
    assert "kernels" not in back and "other_configs" not in back and "compact_mg_table4" not in back


def test_headline_drops_optional_parts_before_growing_past_the_limit():
    import bench
    full = _full_record()
    full["config"]["workload"] = "w" * 1500
    line = bench.headline(full, "/tmp/" + "d" * 400)
    assert len(json.dumps(line)) <= bench.HEADLINE_MAX_BYTES
    assert "value" in line and "roofline" in line and "e2e" in line


def test_details_file_round_trips(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("BENCH_DETAILS_DIR", str(tmp_path))
    full = _full_record()
    path = bench.write_details(full)
    assert path and os.path.dirname(path) == str(tmp_path)
    assert json.load(open(path))["kernels"].keys() == full["kernels"].keys()
