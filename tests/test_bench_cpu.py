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


def test_oracle_sample_takes_a_round_of_subdomains_even_without_budget():
    sys.path.insert(0, ROOT)
    import bench
    s = bench.oracle_sample(types.SimpleNamespace(workload="square2k", seed=0), 0.0)
    assert 1 <= s["subdomains_sampled"] <= s["K"]
    assert s["per_precond_s"] > 0 and s["t_setup_s"] > 0 and s["per_precond_1thread_s"] > 0
