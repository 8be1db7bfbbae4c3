"""The benchmark's reference arm (the oracle timed on the host cores) runs
without a GPU and prints the contract's line for workloads whose pairs have
mixed lengths or are exact integer convolutions; and its sampler reaches
every pair of a mixed batch."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT


@pytest.mark.parametrize("workload,unit", [("conv4", "conv/s"), ("exact6", "conv/s"), ("serve5", "req/s")])
def test_reference_line(workload, unit):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", workload,
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300,
                       env={**os.environ, "RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == unit and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"]


def test_reference_sampler_reaches_every_pair():
    """Lengths 2^6 and 2^12 mixed: every pair gets sampled outputs, and the
    rate is the pairs over the sum of their scaled times (a pair of 2^12
    costs 4096 times one of 2^6)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1005_1497_gb300 import inputs
    pairs = []
    for i, n in enumerate([64, 4096, 64, 4096]):
        f, g = inputs.pairs(13631489, 1, n, seed=50 + i, dtype=np.uint64)
        pairs.append((f[0], g[0], 13631489, "mod"))
    rate, threads, outputs, _ = bench.oracle_rate_mixed(pairs, 0.5)
    assert threads >= 1 and outputs >= 4 * 8
    # the two long pairs dominate: the rate is below what the short ones alone allow
    short_only, _, _, _ = bench.oracle_rate_mixed([pairs[0], pairs[2]], 0.5)
    assert 0 < rate < short_only
