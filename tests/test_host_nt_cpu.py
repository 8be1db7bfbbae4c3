"""The library's host number theory (the plan's validation and tables: Sec. I,
Sec. III-A Prop. 2, Appendix A), compiled on the host from its header and
checked without a GPU against the oracle's independent routines and exact
integer arithmetic: primality (Miller-Rabin against trial division, plus
Carmichael numbers, strong pseudoprimes and a Lucas-Lehmer-proved Mersenne
prime), the order of 2, modular powers, the doubling sequence of the
twiddle tables, Shoup quotients, inverses modulo 2^B and bit reversal."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from conftest import ROOT

TABLE1 = [641, 2424833, 319489, 13631489]
CANDIDATES = [13631489, 26017793, 6700417, 2424833, 974849, 319489, 274177, 114689, 641, 70525124609,
              167772161, 1214251009, 825753601, 63766529, 45592577]


@pytest.fixture(scope="module")
def nt(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("nt") / "nt_host_harness")
    subprocess.check_call([cxx, "-O2", "-std=c++17", os.path.join(ROOT, "tests", "nt_host_harness.cpp"), "-o", exe])

    def run(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        out = r.stdout.strip().split("\n")
        assert len(out) == len(lines)
        return out
    return run


def lucas_lehmer(p):
    """2^p - 1 is prime iff s_(p-2) = 0 for s_0 = 4, s_(i+1) = s_i^2 - 2 mod 2^p - 1 (p an odd prime)."""
    M, s = (1 << p) - 1, 4
    for _ in range(p - 2):
        s = (s * s - 2) % M
    return s == 0


def test_primality(nt, orc):
    rng = np.random.default_rng(1)
    small = [0, 1, 2, 3, 4, 5, 9, 25, 49, 121, 7 * 7 * 7, 65537, 65535, (1 << 31) - 1, 4294967297] + TABLE1 + CANDIDATES
    small += [int(v) for v in rng.integers(2, 1 << 40, 1500, dtype=np.int64)]
    small += [1048573 * 1048571, 1048573 * 1048573, 999983 * 1000003]          # semiprimes near 2^40
    got = nt([f"prime {n}" for n in small])
    for n, g in zip(small, got):
        assert int(g) == int(orc.is_prime(n)), n
    for p in CANDIDATES:
        assert got[small.index(p)] == "1"
    # Carmichael numbers (Fermat liars to every coprime base) and strong
    # pseudoprimes to base 2, each with its factorization
    composites = {561: (3, 11, 17), 1105: (5, 13, 17), 1729: (7, 13, 19), 41041: (7, 11, 13, 41),
                  825265: (5, 7, 17, 19, 73), 321197185: (5, 19, 23, 29, 37, 137), 2047: (23, 89),
                  3277: (29, 113), 4033: (37, 109), 4681: (31, 151), 8321: (53, 157),
                  # a strong pseudoprime to all prime bases up to 23
                  3825123056546413051: (149491, 747451, 34233211)}
    for n, fac in composites.items():
        assert math.prod(fac) == n and all(orc.is_prime(f) for f in fac)
    got = nt([f"prime {n}" for n in composites])
    assert got == ["0"] * len(composites)
    # Mersenne primes proved by Lucas-Lehmer; 2^59 - 1 is composite
    for p in (31, 61):
        assert lucas_lehmer(p)
    assert not lucas_lehmer(59)
    assert nt([f"prime {(1 << 31) - 1}", f"prime {(1 << 61) - 1}", f"prime {(1 << 59) - 1}"]) == ["1", "1", "0"]


def test_order_of_two(nt, orc):
    primes = [7, 11, 17, 31, 97, 257, 65537] + TABLE1 + CANDIDATES
    got = nt([f"order {m}" for m in primes])
    for m, g in zip(primes, got):
        o = orc.order(2, m, 1 << 26)
        assert o > 0
        want = o if o & (o - 1) == 0 else 0         # a power of two, else not a Rader prime: 0
        assert int(g) == want, m
    # Table 1 orders and the 64-bit prime's
    assert [int(g) for g in nt([f"order {m}" for m in TABLE1 + [70525124609]])] == \
        [1 << 6, 1 << 10, 1 << 12, 1 << 19, 1 << 20]


def test_pow_and_doubling(nt, orc):
    rng = np.random.default_rng(2)
    cases = []
    for _ in range(300):
        m = int(rng.integers(2, 1 << 62, dtype=np.int64))
        cases.append((int(rng.integers(0, 1 << 62, dtype=np.int64)), int(rng.integers(0, 1 << 62, dtype=np.int64)), m))
    got = nt([f"pow {a} {e} {m}" for a, e, m in cases])
    for (a, e, m), g in zip(cases, got):
        assert int(g) == pow(a, e, m) == orc.mod_pow(a, e, m)
    for m in (641, 65537, 13631489, 70525124609):
        count = 1500
        seq = [int(v) for v in nt([f"powers {count} {m}"])[0].split()]
        assert seq == [orc.mod_pow(2, k, m) for k in range(count)], m


def test_shoup_shift_inverse_brv(nt):
    rng = np.random.default_rng(3)
    lines, want = [], []
    for m in (641, 13631489, 70525124609, (1 << 57) - 13):
        for B in (32, 64):
            if B == 32 and m >= 1 << 31:
                continue
            for z in [0, 1, m - 1] + [int(v) for v in rng.integers(0, m, 20, dtype=np.int64)]:
                lines.append(f"shoupq {z} {m} {B}")
                want.append((z << B) // m)
                lines.append(f"shl {z} {B} {m}")
                want.append((z << B) % m)
    for m in [1, 3, 641, 13631489, 70525124609] + [int(v) | 1 for v in rng.integers(1, 1 << 62, 50, dtype=np.int64)]:
        for B in (32, 64):
            lines.append(f"invpow2 {m} {B}")
            want.append(pow(m, -1, 1 << B))
    for bits in (1, 5, 10, 14, 19, 20):
        for i in [0, 1, (1 << bits) - 1] + [int(v) for v in rng.integers(0, 1 << bits, 10)]:
            lines.append(f"brv {i} {bits}")
            want.append(int(format(i, f"0{bits}b")[::-1], 2))
    got = [int(g) for g in nt(lines)]
    for line, g, w in zip(lines, got, want):
        assert g == w, line
