"""The convolution server's admission pool (first fit over one device region,
256-byte granules, coalescing on release), compiled on the host and driven
without a GPU: fragmentation and coalescing cases, and long random
sequences checked against a reference model and the allocator's
invariants (allocations disjoint and inside the region, free blocks never
adjacent, a failure only when no free block is large enough)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from conftest import ROOT

G = 256


@pytest.fixture(scope="module")
def pool_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("pool") / "pool_harness")
    subprocess.check_call([cxx, "-O2", "-std=c++17", os.path.join(ROOT, "tests", "pool_harness.cpp"), "-o", exe])
    return exe


def run(exe, lines):
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    out = r.stdout.strip().split("\n")
    assert len(out) == len(lines)
    return out


class Model:
    """First fit over a sorted free list of (offset, size); release merges
    with both neighbours."""

    def __init__(self, size):
        self.free = [(0, size)]
        self.size, self.used, self.peak = size, 0, 0

    @staticmethod
    def rnd(b):
        return (b + G - 1) // G * G

    def alloc(self, b):
        b = self.rnd(b)
        for i, (o, s) in enumerate(self.free):
            if s >= b:
                self.free[i:i + 1] = [(o + b, s - b)] if s > b else []
                self.used += b
                self.peak = max(self.peak, self.used)
                return o
        return -1

    def release(self, o, b):
        b = self.rnd(b)
        self.used -= b
        self.free.append((o, b))
        self.free.sort()
        merged = []
        for fo, fs in self.free:
            if merged and merged[-1][0] + merged[-1][1] == fo:
                merged[-1] = (merged[-1][0], merged[-1][1] + fs)
            else:
                merged.append((fo, fs))
        self.free = merged


def test_fragmentation_and_coalescing(pool_exe):
    lines = ["init 4096"] + ["alloc 256"] * 16 + ["alloc 1"]
    out = run(pool_exe, lines)
    assert [int(v) for v in out[1:17]] == [256 * i for i in range(16)]
    assert out[17] == "-1"                                   # full
    # free every other block: 2 KB free in total, but no 512-byte hole
    lines = ["init 4096"] + ["alloc 256"] * 16 + [f"free {256 * i} 256" for i in range(0, 16, 2)] + ["alloc 512"]
    assert run(pool_exe, lines)[-1] == "-1"
    # freeing block 1 joins blocks 0..2 into one hole at offset 0
    assert run(pool_exe, lines[:-1] + ["free 256 256", "alloc 768", "alloc 256"])[-2:] == ["0", "1024"]
    # everything released in reverse order coalesces back to the whole region
    lines = ["init 4096"] + ["alloc 1000"] * 4 + [f"free {1024 * i} 1000" for i in range(3, -1, -1)] + ["alloc 4096"]
    out = run(pool_exe, lines)
    assert [int(v) for v in out[1:5]] == [0, 1024, 2048, 3072] and out[-1] == "0"
    # granules: 1 byte takes 256, 257 bytes take 512
    assert run(pool_exe, ["init 4096", "alloc 1", "alloc 257", "alloc 1", "peak"])[1:] == ["0", "256", "768", "1024"]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_against_model(pool_exe, seed):
    rng = np.random.default_rng(seed)
    size = 1 << 20
    model = Model(size)
    live = {}
    lines, expect = ["init %d" % size], ["ok"]
    for _ in range(3000):
        if live and (rng.random() < 0.45 or model.used > 0.9 * size):
            off = list(live)[int(rng.integers(0, len(live)))]
            b = live.pop(off)
            model.release(off, b)
            lines.append(f"free {off} {b}")
            expect.append("ok")
        else:
            b = int(rng.integers(1, 64 * 1024))
            off = model.alloc(b)
            lines.append(f"alloc {b}")
            expect.append(str(off))
            if off >= 0:
                live[off] = b
            else:                                            # first fit fails only without a large enough hole
                assert all(s < Model.rnd(b) for _, s in model.free)
        # invariants of the model's state
        blocks = sorted((o, Model.rnd(b)) for o, b in live.items())
        for (o1, s1), (o2, _) in zip(blocks, blocks[1:]):
            assert o1 + s1 <= o2
        assert all(0 <= o and o + s <= size for o, s in blocks)
        assert all(a[0] + a[1] < b[0] for a, b in zip(model.free, model.free[1:]))
        assert model.used + sum(s for _, s in model.free) == size
    lines.append("peak")
    expect.append(str(model.peak))
    assert run(pool_exe, lines) == expect
