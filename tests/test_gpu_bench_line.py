"""bench.py's default run on the GPU prints one JSON line that carries the
headline workload and, under "configs", the single, large, uneven and
serving workloads, each with its rate, roofline, clocks, end-to-end rate and
CPU baseline (a short run: few steps, a small CPU budget)."""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_default_line_carries_every_workload():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3", "--warmup", "3",
                        "--cpu-seconds", "2"], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "clocks", "e2e", "gpu_launches"):
        assert k in d, k
    assert d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["gpu_launches"] >= 3
    rf = d["roofline"]
    assert rf["bound"] == "alu" and 0 < rf["frac"] < 1.2 and rf["achieved"] > 0 and rf["peak"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "single_thread" in d["cpu_baseline"] and "direct" in d["cpu_baseline"]
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["e2e"]["bit_identical_to_device_path"] is True
    assert d["plain_form"]["bit_identical_to_fused"] is True
    cfg = d["configs"]
    assert set(cfg) == {"conv1", "conv3", "conv4", "serve5"}
    for name, c in cfg.items():
        for k in ("value", "unit", "ms_per_step", "config", "roofline", "clocks", "e2e", "cpu_baseline"):
            assert k in c, (name, k)
        assert c["value"] > 0 and c["cpu_baseline"]["value"] > 0, name
    assert cfg["serve5"]["latency_us"]["p50"] <= cfg["serve5"]["latency_us"]["p99"]
    assert cfg["serve5"]["capacity"]["req_per_s"] > 0
    assert cfg["conv3"]["e2e"]["bit_identical_to_device_path"] is True
    assert cfg["conv4"]["e2e"]["bit_identical_to_device_path"] is True
    assert cfg["conv3"]["noalloc"]["bit_identical"] is True
