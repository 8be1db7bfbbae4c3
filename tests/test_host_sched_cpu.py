"""The library's host scheduling rules (csrc/host_sched.h), compiled on the
host and checked without a GPU: which batches of the one-warp lengths run one
thread block per pair (the limit is where the measured crossover on GB300
lies: 608 pairs of 2^10 with 32-bit words on 152 SMs), and how the
host-buffer pipeline cuts a batch into chunks (every pair covered exactly
once, in order; no chunk above the staging slot; the shrinking last chunks
only where they were measured to help)."""
import os
import random
import shutil
import subprocess

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def hs(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("hs") / "host_sched_harness")
    subprocess.check_call([cxx, "-O2", "-std=c++17", os.path.join(ROOT, "tests", "host_sched_harness.cpp"), "-o", exe])

    def run(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        out = r.stdout.strip("\n").split("\n")
        assert len(out) == len(lines)
        return out
    return run


def test_small_batch_limit(hs):
    cases = {(10, 10, 4, 152): 608, (9, 10, 4, 152): 1216, (8, 10, 4, 152): 2432, (6, 10, 4, 152): 4864,
             (0, 10, 4, 152): 4864, (9, 9, 8, 152): 608, (7, 9, 8, 152): 2432, (11, 10, 4, 152): 0,
             (10, 9, 8, 152): 0, (10, 10, 4, 1): 4, (10, 10, 8, 1): 2, (10, 10, 4, 0): 0}
    got = hs([f"small {L} {rw} {wb} {n}" for (L, rw, wb, n) in cases])
    assert [int(x) for x in got] == list(cases.values())
    # never below one pair for a one-warp length, never above 32 pairs per SM,
    # and non-increasing in the length
    for wb, rw in ((4, 10), (8, 9)):
        for nsm in (1, 8, 132, 152, 160):
            vals = [int(x) for x in hs([f"small {L} {rw} {wb} {nsm}" for L in range(0, rw + 1)])]
            assert all(1 <= v <= 32 * nsm for v in vals)
            assert all(a >= b for a, b in zip(vals, vals[1:]))


def test_chunk_pairs(hs):
    cases = {(65536, 0, 4096): 384, (65536, 1, 4096): 256, (2 << 20, 1, 64): 8, (4096, 0, 3): 3,
             (1 << 30, 0, 10): 1, (1 << 30, 1, 1): 1, (8, 0, 10 ** 9): (48 << 20) // 16}
    got = hs([f"chunkpairs {s} {sp} {b}" for (s, sp, b) in cases])
    assert [int(x) for x in got] == list(cases.values())


def sizes(hs, pairs, chunk, shrink):
    out = hs([f"chunks {pairs} {chunk} {int(shrink)}"])[0]
    return [] if out == "-" else [int(x) for x in out.split()]


def test_chunk_sizes_examples(hs):
    # the headline batch: nine full chunks, a ragged one, then 1/2, 1/4, 1/8
    assert sizes(hs, 4096, 384, True) == [384] * 9 + [304, 192, 96, 48]
    assert sizes(hs, 2000, 384, True) == [384] * 4 + [128, 192, 96, 48]
    assert sizes(hs, 1100, 384, True) == [384, 384, 332]          # fewer than four full chunks: no tail
    assert sizes(hs, 64, 8, False) == [8] * 8                       # the split path keeps full chunks
    assert sizes(hs, 64, 8, True) == [8] * 7 + [1, 4, 2, 1]
    assert sizes(hs, 4096, 7, True) == [7] * 585 + [1]             # chunks below 8 pairs: no tail
    assert sizes(hs, 5, 7, True) == [5]
    assert sizes(hs, 0, 8, True) == []


def test_chunk_sizes_cover_every_pair_once(hs):
    rng = random.Random(7)
    for _ in range(300):
        chunk = rng.choice([1, 2, 7, 8, 9, 64, 256, 384, 1000])
        pairs = rng.randrange(0, 12 * chunk + 5)
        shrink = rng.random() < 0.5
        v = sizes(hs, pairs, chunk, shrink)
        assert sum(v) == pairs and all(0 < c <= chunk for c in v)
        tail = shrink and chunk >= 8 and pairs >= 4 * chunk
        if tail:
            assert v[-3:] == [chunk // 2, chunk // 4, chunk // 8]
        else:
            assert all(c == chunk for c in v[:-1])
