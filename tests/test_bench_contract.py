"""The benchmark's reference arm runs the oracle on the host cores (no GPU) and prints one JSON
line with the fields the benchmark contract names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "20000",
                          "--per-sigma", "3", "--steps", "1", "--warmup", "0"],
                         check=True, capture_output=True, text=True, cwd=ROOT, timeout=600).stdout
    lines = [ln for ln in out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "queries/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "20000",
                          "--per-sigma", "3", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert res.returncode == 0 and res.stdout.strip() == ""


def test_dram_traffic_only_for_the_sizes_and_source_it_was_taken_on():
    sys.path.insert(0, ROOT)
    import bench
    table = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, entry in table.items():
        kernel, _, qt = key.partition("@qt")
        wl = dict(entry.get("workload", {}))
        wl.setdefault("queries", 3000)
        got = bench.traffic_for(kernel, int(qt or 0), wl)
        assert got is None or abs(got - entry["bytes_per_launch"] * entry.get("scale", 1.0)) < 1.0
        assert bench.traffic_for(kernel, int(qt or 0), dict(wl, n=wl.get("n", 0) + 16)) is None
