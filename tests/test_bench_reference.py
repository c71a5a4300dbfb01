"""CPU test of bench.py's reference arm (the oracle timed on the host on a
bounded sample of the benchmark workload): it needs no GPU, prints one JSON
line with the contract's keys, and under a multi-rank launch only rank 0
prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline",
        "e2e"}


def run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--sample-points", "1", *args],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_contract_line():
    lines = run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["unit"] == "resolvent columns/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "grid5pt_rational_n40000_bw200_N64_L32"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_only_rank_zero_prints():
    assert run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_cpu_baseline_reports_one_core_and_all_cores_runs():
    sys.path.insert(0, ROOT)
    import bench
    d = bench.cpu_baseline(40, 2)
    assert d["kind"] == "oracle" and d["cores"] == 1 and d["value"] > 0 and d["cpu"]
    par = d["parallel"]
    assert 1 <= par["cores"] <= 16 and par["value"] > 0
    assert f"{par['cores']} sampling points" in par["sample"]
