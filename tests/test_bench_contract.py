"""The benchmark's output contract, on CPU: the reference arm (the oracle on
the host cores) prints one JSON line with the required keys, and the
committed ncu summaries carry the figures the GPU arm reads from them."""
import json
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
         "--warmup", "1", "--workload", "tiny"],
        capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "Gbps" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_profiles_carry_the_figures_bench_reads():
    sys.path.insert(0, ROOT)
    import bench
    for name in ("pfac_scan_paper_scale.md", "pfac_scan_acgt.md"):
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        assert re.search(r"dram_bytes_per_launch_full_size:\s*[0-9.]+", txt), name
        assert re.search(r"kernel_source_sha256:\s*[0-9a-f]{64}", txt), name
        assert "ncu --metrics gpu__time_duration.sum --clock-control none" in txt
        assert "ncu --set full --clock-control none" in txt
    assert len(bench.kernel_source_sha()) == 64
