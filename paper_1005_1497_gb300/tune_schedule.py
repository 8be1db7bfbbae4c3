"""Autotune the convolution schedule of this GPU and save it as JSON.

    python -m paper_1005_1497_gb300.tune_schedule [--out PATH]

Runs ``ntt_autotune`` for every length of the two moduli the library's
workloads use -- m = 13631489 (32-bit words, N = 2^6 .. 2^19) and the
64-bit-word prime 70525124609 (N = 2^8 .. 2^18) -- and writes the recorded
table (one entry per GPU name, word size and log2 N: split-path wave and
form, whole-sequence threads per block, persistent-launch membership).
``bench.py`` loads the packaged GB300 file instead of tuning inside its
timed run; plans made after ``ntt_autotune_load`` follow it.

The batch of each trial: 32-bit lengths get the pair count an uneven batch
of 10,000 pairs over 2^6 .. 2^19 holds per length (about 714), 64-bit
lengths 64 pairs (serving batches are small).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "schedules", "gb300.json")

M32, M64 = 13631489, 70525124609


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--pairs32", type=int, default=714)
    ap.add_argument("--pairs64", type=int, default=64)
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1005_1497_gb300 import ntt

    results = []
    for m, lo, hi, pairs in ((M32, 6, 19, a.pairs32), (M64, 8, 18, a.pairs64)):
        for L in range(lo, hi + 1):
            r = ntt.ntt_autotune(m, 1 << L, pairs)
            r.update({"m": m, "log2N": L, "pairs": pairs})
            results.append(r)
            print(json.dumps(r), flush=True)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    ntt.ntt_autotune_save(a.out)
    print(f"wrote {a.out} ({len(results)} entries)", flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
