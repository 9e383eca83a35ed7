"""bench.py keeps its output contract: one JSON line with the keys and types the
measurement reports (metric, value, unit, timing, e2e, roofline, cpu_baseline,
clocks, launches), for the GPU arm and for the reference arm (the oracle).

CPU: the reference arm (one bounded oracle window).
GPU: the GPU arm on the bench workload with the side measurements switched off.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, timeout=900):
    r = subprocess.run([sys.executable, "bench.py"] + list(args), cwd=ROOT, capture_output=True, text=True,
                       timeout=timeout)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-3000:]
    return json.loads(lines[0])


def _common(d, steps, warmup):
    assert d["metric"] and d["unit"] == "cell-updates/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (steps, warmup, 1)
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["data"] == "synthetic"
    assert d["dtype"] == "f64" and d["vs_baseline"] is None
    assert "workload" in d["config"]
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] >= 0 and e["d2h_bytes_per_step"] >= 0
    cb = d["cpu_baseline"]
    assert cb["value"] > 0 and cb["cores"] >= 1 and cb["kind"] == "oracle" and cb["sample"]


def test_reference_arm_line():
    d = _bench("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference"
    _common(d, 1, 0)
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_gpu_arm_line():
    d = _bench("--steps", "1", "--warmup", "3", "--no-sizes", "--no-2d", "--no-batch", "--no-adjoint", "--no-fp32")
    assert "impl" not in d or d["impl"] != "reference"
    _common(d, 1, 3)
    assert d["gpu_launches"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == d["e2e"]["d2h_bytes_per_step"] == d["config"]["n"] * 8
    rf = d["roofline"]
    assert rf["bound"] in ("hbm", "tensor", "alu") and rf["unit"] in ("GB/s", "TFLOP/s")
    assert rf["achieved"] > 0 and rf["peak"] > 0 and abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    assert rf["traffic"] is None or rf["traffic"] > 0
    ck = d["clocks"]
    assert ck["sm_mhz"] > 0 and ck["sm_max_mhz"] > 0 and isinstance(ck["reasons"], list)
    assert d["classic"]["value"] > 0 and d["speedup_vs_classic"] > 0
