"""The integer-pipe rates behind the benchmark's integer roofline: 32-bit
multiply-adds issue at 64 per clock per SM, the high half of a product
(umulhi) at half that rate, so a Shoup product (umulhi + two multiplies)
takes four multiply-add issue slots.  The probe kernels are plain
independent chains (tests/int_pipes_probe.cu); this test builds and runs
them and checks the rates against those unit counts (at the clock the GPU
reports as its maximum; a GPU held below it reads low, hence the margins).

    python -m pytest tests/test_gpu_int_pipes.py -m gpu -s     (prints the rates)
"""
import os
import shutil
import subprocess

import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


def test_integer_pipe_rates(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = str(tmp_path / "int_pipes_probe")
    subprocess.run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "int_pipes_probe.cu")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120, check=True).stdout
    print(out)
    vals = {}
    for line in out.splitlines():
        k, _, v = line.partition(" ")
        vals[k] = v
    assert vals["status"] == "no error"
    sms, hz = int(vals["sms"]), int(vals["clock_khz"]) * 1e3
    imad = float(vals["imad_per_s"]) / sms / hz              # per SM per clock
    mulhi = float(vals["umulhi_per_s"]) / sms / hz
    shoup = float(vals["shoup_per_s"]) / sms / hz
    assert 48 <= imad <= 66, imad                            # 64 lanes per SM per clock
    assert 0.4 <= mulhi / imad <= 0.6, (mulhi, imad)         # half rate: two issue slots
    assert 0.2 <= shoup / imad <= 0.3, (shoup, imad)         # four slots per Shoup product
