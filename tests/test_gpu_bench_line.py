"""The JSON line of bench.py on one GPU (a short run without the extra sections): the keys of
the benchmark contract with values of the right kind, the roofline's figures consistent with
the line's own time, and the end-to-end figure with its copied bytes."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_keys_and_roofline():
    cmd = [sys.executable, "bench.py", "--steps", "5", "--warmup", "3", "--no-variants", "--no-extras",
           "--no-cpu-baseline", "--clock-window", "0"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["unit"] == "MLUPS" and d["n_gpus"] == 1 and d["steps"] == 5 and d["warmup"] >= 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["gpu_launches"] == 5
    assert "workload" in d["config"]
    sites = d["config"]["Lx"] * d["config"]["Lz"]
    assert d["value"] == pytest.approx(sites / (d["ms_per_step"] * 1e-3) / 1e6, rel=1e-9)
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["bytes_per_site"] == 592
    assert r["achieved"] == pytest.approx(592 * sites / (d["ms_per_step"] * 1e-3) / 1e9, rel=1e-9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-12)
    assert 0.3 < r["frac"] < 1.1
    sec = r["secondary"]
    assert sec["bound"] == "fp64_pipe" and sec["instr_per_site"] == 42 and 0.1 < sec["frac"] < 1.2
    e = d["e2e"]
    assert e["unit"] == "MLUPS" and 0 < e["value"] < d["value"]
    assert e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == 37 * 8 * sites
