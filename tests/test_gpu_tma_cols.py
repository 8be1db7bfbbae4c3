"""The split path's column passes staged through shared memory by the TMA
unit (tests/tma_cols_probe.cu): tiled tensor copies (cp.async.bulk.tensor)
and untiled row copies (cp.async.bulk), producer/consumer mbarrier
pipelines, against the library's plain column kernels on the same inputs.
Every staged kernel must give the plain kernels' words exactly and no wait
may run out; the times are printed (they are the evidence for keeping the
plain kernels, not a pass condition).

    python -m pytest tests/test_gpu_tma_cols.py -m gpu -s     (prints the times)
"""
import os
import shutil
import subprocess

import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


def test_staged_column_passes_equal_the_plain_ones(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = str(tmp_path / "tma_cols_probe")
    subprocess.run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_1005_1497_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-o", exe, os.path.join(HERE, "tma_cols_probe.cu"), "-lcuda"], check=True)
    out = subprocess.run([exe, "16", "3"], capture_output=True, text=True, timeout=300, check=True).stdout
    print(out)
    lines = out.strip().splitlines()
    assert lines[-1] == "status no error", out
    rows = [ln.split() for ln in lines[:-1]]
    staged = [r for r in rows if not r[0].startswith("plain")]
    assert len(staged) == 6, out
    for name, threads, per_sm, ms, diff, err in staged:
        assert int(per_sm) >= 1 and float(ms) > 0, name
        assert int(diff) == 0 and int(err) == 0, (name, diff, err)
