"""CPU-only checks of the C ABI: the library loads, exports every function the
header declares, and the host-side plan validation rejects bad parameters
before touching a GPU."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "ntt_gb300.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_0-9]+)\s*\([^;{]*\)\s*;", src)) - {"sizeof"})


@pytest.fixture(scope="module")
def ntt():
    from paper_1005_1497_gb300 import build, ntt as mod
    build.build()
    return mod


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ntt_plan", "ntt_forward", "ntt_inverse", "conv_circular", "conv_batched", "ntt_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol(ntt):
    so = ctypes.CDLL(ntt.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert missing == []
    assert set(_declared()) == set(ntt.SIGNATURES)


def test_status_strings(ntt):
    lib = ntt.lib()
    for code, name in ntt.STATUS.items():
        assert lib.ntt_status_str(code).decode() == name


@pytest.mark.parametrize("m,N,status", [
    (341, 8, 2),            # Sec. II: 341 = 11 * 31 is composite
    (13631487, 8, 2),       # composite neighbour
    (7, 2, 2),              # ord_7(2) = 3 is not a power of two (Fig. 1 (c))
    (13631489, 3, 1),       # not a power of two
    (13631489, 1 << 20, 1), # does not divide ord = 2^19 (Sec. I)
    (641, 128, 1),          # Table 1: 641 allows N <= 64
    (2424833, 2048, 1),     # Table 1: N_Max = 1024
    (13631489, 0, 1),
])
def test_plan_rejects(ntt, m, N, status):
    h = ctypes.c_void_p()
    assert ntt.lib().ntt_plan(m, N, ctypes.byref(h)) == status
    assert not h.value
    assert ntt.lib().ntt_last_error().decode()


def test_null_arguments(ntt):
    lib = ntt.lib()
    assert lib.ntt_plan(13631489, 8, None) == 8
    assert lib.ntt_forward(None, None, None, 1, None) == 8
    assert lib.conv_circular(None, None, None, None, 1, None) == 8
    assert lib.conv_batched(13631489, None, 0, None) == 8


def test_torch_generator_matches_numpy():
    """The device-side generator used by the benchmark gives the same values
    as the host generator used by the oracle tests."""
    import numpy as np
    import torch

    from paper_1005_1497_gb300 import inputs
    for m in (13631489, 641, 70525124609):
        a = inputs.uniform_mod(m, 5000, seed=11, stream=3, start=777, dtype=np.uint64)
        b = inputs.uniform_mod_torch(m, 5000, seed=11, stream=3, start=777, device="cpu", dtype=torch.int64)
        assert np.array_equal(a, b.numpy().astype(np.uint64))


@pytest.mark.parametrize("N,bits,status", [
    (3, 20, 1),             # not a power of two
    (0, 20, 1),
    (1024, 0, 4),           # bound outside 1..63: outputs are signed 64-bit
    (1024, 64, 4),
])
def test_exact_plan_rejects(ntt, N, bits, status):
    h = ctypes.c_void_p()
    assert ntt.lib().ntt_exact_plan(N, bits, ctypes.byref(h)) == status
    assert not h.value
    assert ntt.lib().ntt_exact_plan(1024, 20, None) == 8
    assert ntt.lib().conv_exact(None, None, None, None, 1, None) == 8


def test_exact_candidate_primes_are_fermat_factors(orc):
    """Every prime the exact convolution may use is a prime factor of the
    Fermat number its table entry names, so ord_p(2) = 2^(n+1) (Sec. III-A)."""
    import re
    src = open(os.path.join(ROOT, "paper_1005_1497_gb300", "csrc", "ntt_exact.cu")).read()
    table = src[src.index("kCandidates[]"):]
    table = table[:table.index("};")]
    rows = re.findall(r"(\d+)ull,\s*//\s*F_(\d+)", table)
    assert len(rows) >= 10
    for p, n in rows:
        p, n = int(p), int(n)
        assert orc.is_prime(p), p
        assert pow(2, 1 << n, p) == p - 1, (p, n)          # p | F_n = 2^(2^n) + 1
        assert orc.order(2, p) == 1 << (n + 1), (p, n)


@pytest.mark.parametrize("m,N,mode,status", [
    (13631489, 64, 0, 2),   # not a factor of F_4 or F_5
    (4294967297, 64, 0, 2), # F_5 itself is composite
    (641, 128, 0, 1),       # ord_641(2) = 64
    (65537, 64, 0, 1),      # ord_65537(2) = 32
    (641, 48, 0, 1),        # not a power of two
    (641, 64, 2, 8),        # unknown mode
])
def test_shift_rejects(ntt, m, N, mode, status):
    buf = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    assert ntt.lib().conv_circular_shift(m, N, buf, buf, buf, 1, mode, None) == status


def test_launch_counter_needs_no_gpu(ntt):
    a = ntt.launch_count()
    assert isinstance(a, int) and a >= 0
    assert ntt.launch_count() >= a


def test_schedule_file_roundtrip_without_a_gpu(ntt, tmp_path):
    """ntt_autotune_load / _save on the host: entries of the current format and
    older entries without block / persist (which take the defaults) are read,
    malformed ones are skipped, and saving writes every knob back."""
    src = tmp_path / "in.json"
    src.write_text('{"schedules": [\n'
                   '  {"gpu": "Some GPU", "word_bits": 32, "log2N": 12, "wave": 0, "twist": 1, "block": 256, '
                   '"persist": 1, "ms": 0.5},\n'
                   '  {"gpu": "Some GPU", "word_bits": 32, "log2N": 17, "wave": 12, "twist": 0, "ms": 0.25},\n'
                   '  {"gpu": "Some GPU", "word_bits": 64, "log2N": 9, "wave": 0, "twist": 1, "ms": 0.1},\n'
                   '  {"gpu": "Some GPU", "word_bits": 32, "log2N": 13, "wave": 0, "twist": 1, "block": 300, '
                   '"persist": 0, "ms": 1.0}\n'
                   ']}\n')
    ntt.ntt_autotune_load(str(src))
    out = tmp_path / "out.json"
    ntt.ntt_autotune_save(str(out))
    rows = {(r["word_bits"], r["log2N"]): r for r in
            (__import__("json").loads(ln.strip().rstrip(",")) for ln in open(out) if '"gpu"' in ln)}
    assert set(rows) >= {(32, 12), (32, 17), (64, 9)} and (32, 13) not in rows     # block 300 is not a choice
    assert (rows[(32, 12)]["block"], rows[(32, 12)]["persist"]) == (256, 1)
    assert (rows[(32, 17)]["wave"], rows[(32, 17)]["twist"], rows[(32, 17)]["block"]) == (12, 0, 512)
    assert rows[(32, 17)]["persist"] == 0 and rows[(64, 9)]["persist"] == 1       # defaults: one-warp lengths persist
    with pytest.raises(ntt.NttError):
        bad = tmp_path / "bad.json"
        bad.write_text('{"schedules": []}\n')
        ntt.ntt_autotune_load(str(bad))


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has, in the C header compiled as plain
    C, the same size and the same offset for every field as its ctypes twin
    (a stale mirror would hand the library shifted fields)."""
    import shutil
    import subprocess

    from paper_1005_1497_gb300 import ntt as mod

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    pairs = [("ntt_plan_info_t", mod.PlanInfo), ("ntt_exact_info_t", mod.ExactInfo), ("ntt_conv_desc", mod.ConvDesc),
             ("ntt_server_config", mod.ServerConfig), ("ntt_server_stats", mod.ServerStats),
             ("ntt_tune_result", mod.TuneResult)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ntt_gb300.h"', "int main(void) {"]
    want = []
    for cname, py in pairs:
        lines.append(f'    printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(py))
        for fname, _ in py._fields_:
            lines.append(f'    printf("%zu\\n", offsetof({cname}, {fname}));')
            want.append(getattr(py, fname).offset)
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe])
    got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert got == want
