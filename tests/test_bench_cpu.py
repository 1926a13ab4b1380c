"""The benchmark's CPU legs (the oracle arm and the CPU-baseline sample) run without a GPU."""
import json
import os
import subprocess
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "square2k",
                          "--steps", "1", "--warmup", "0", "--cpu-seconds", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["unit"] == "solves/s" and rec["higher_is_better"] is True
    assert rec["value"] > 0 and rec["steps"] == 1 and rec["warmup"] == 0
    assert rec["config"]["workload"] == "square2k"
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == rec["value"] and cb["cores"] >= 1 and cb["sample"]
    assert 0 < cb["value_1thread"] <= cb["value"] * 1.5 and cb["cpu_model"] and cb["nproc"] >= 1
    assert rec["e2e"] == {"value": rec["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    # the printed steps are the samples that ran: their wall time, not the extrapolated solve
    ex = rec["extrapolated"]
    assert ex["steps_run"] == 1 and ex["solve_s"] > 0 and abs(1.0 / ex["solve_s"] - rec["value"]) < 1e-9 * rec["value"]
    assert 0 < rec["ms_per_step"] < 600e3


def test_oracle_gnn_sample_takes_a_round_of_subdomains_even_without_budget():
    sys.path.insert(0, ROOT)
    import bench
    a = types.SimpleNamespace(workload="square2k", seed=0)
    pool = bench._one_thread_pool(2)
    try:
        s = bench.oracle_gnn_sample(a, pool, 2, 0.0)
    finally:
        pool.terminate()
        pool.join()
    assert s["subdomains_sampled"] == 2 and s["K"] == 4
    assert s["dss_app_s"] > 0 and s["t_setup_s"] > 0 and s["dss_app_1thread_s"] > 0
    assert s["t_coarse_s"] > 0 and s["t_fcg_iter_s"] > 0
    assert bench.gnn_solve_seconds(s, 10) > bench.gnn_solve_seconds(s, 1) > s["t_setup_s"]


def test_oracle_lu_baseline_runs_whole_solves_on_the_small_workload():
    """square2k: the oracle's DDM-LU PCG converges within the budget, so the baseline is a
    measured whole solve (not extrapolated), alone and as replicas on two cores."""
    sys.path.insert(0, ROOT)
    import bench
    a = types.SimpleNamespace(workload="square2k", seed=0, tol=1e-6, cpu_seconds=60.0)
    b = bench.oracle_lu_baseline(a, lu_iterations=20, replicas=2)
    assert b["kind"] == "oracle" and not b["extrapolated"] and b["cores"] in (1, 2)
    assert b["value"] > 0 and b["value_1thread"] > 0 and b["iterations"] > 0
    assert abs(b["value_1thread"] - 1.0 / b["solve_s_1thread"]) < 1e-12 * b["value_1thread"]


def test_lu_solve_seconds_scales_a_sampled_run():
    sys.path.insert(0, ROOT)
    import bench
    r = {"converged": False, "t_setup_s": 2.0, "iterations_run": 4, "t_iterations_s": 1.0}
    assert bench._lu_solve_seconds(r, 40) == (12.0, 40)
    r = {"converged": True, "t_setup_s": 2.0, "iterations_run": 17, "t_iterations_s": 3.0}
    assert bench._lu_solve_seconds(r, 40) == (5.0, 17)
