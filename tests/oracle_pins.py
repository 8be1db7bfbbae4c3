"""Pins for the CPU oracle: every check compares the oracle with something the
paper prints, a closed form, an invariant, or a brute-force count on tiny
inputs -- never with a retyped copy of its own formula.

``run_pins(o)`` returns the names of the pins that fail, so that the same
suite can be run on the real oracle (no failures allowed) and on deliberately
mutated builds of it (at least one failure required)."""
from __future__ import annotations

import numpy as np

from conftest import golden

M = 13631489                      # Table 1, F_18 row
M64 = 70525124609                 # 33629 * 2^21 + 1, a factor of F_19 (builder's choice)
SMALL = [(17, 8), (641, 64), (2424833, 1024), (319489, 4096), (M, 1 << 19)]


def _rng(seed):
    return np.random.default_rng(seed)


def pin_fig1(o):
    for base, m, seq, nmax in golden("fig1_digital_circles.txt"):
        base, m, nmax = int(base), int(m), int(nmax)
        vals = [int(v) for v in seq.split(",")]
        assert [o.mod_pow(base, i, m) for i in range(len(vals))] == vals
        assert o.order(base, m) == nmax


def pin_table1(o):
    for m, nmax, fermat, word in golden("table1_rader_primes.txt"):
        m, nmax, fermat, word = int(m), int(nmax), int(fermat), int(word)
        assert o.is_prime(m)
        assert o.order(2, m) == nmax
        # m | F_fermat = 2^(2^fermat) + 1  <=>  2^(2^fermat) = -1 (mod m)
        assert o.mod_pow(2, 1 << fermat, m) == m - 1
        assert nmax == 1 << (fermat + 1)          # Prop. 2: order 2^(n+1) for a factor of F_n
        assert m < (1 << word)


def pin_mersenne(o):
    for row in golden("mersenne_factors.txt"):
        n, factors = int(row[0]), [int(v) for v in row[1:]]
        prod = 1
        for p in factors:
            assert o.is_prime(p), p
            prod *= p
            # 2^n = 1 (mod p) so the order of 2 divides n (digital circle)
            assert n % o.order(2, p) == 0
        assert prod == (1 << n) - 1


def pin_carmichael_341(o):
    facts = {r[0]: r[1:] for r in golden("number_facts.txt")}
    m = int(facts["carmichael_modulus"][0])
    p, q = (int(v) for v in facts["carmichael_factors"])
    nu = int(facts["carmichael_nu"][0])
    assert p * q == m and not o.is_prime(m) and o.is_prime(p) and o.is_prime(q)
    assert o.mod_pow(2, nu, m) == 1 and o.mod_pow(2, m - 1, m) == 1
    assert o.order(2, m) == nu
    assert ((1 << nu) - 1) % m == 0


def pin_f5(o):
    facts = {r[0]: r[1:] for r in golden("number_facts.txt")}
    a, b = (int(v) for v in facts["f5_factors"])
    n = int(facts["f5_max_log2"][0])
    assert a * b == (1 << 32) + 1
    for p in (a, b):
        assert o.is_prime(p)
        assert o.order(2, p) == 1 << n
        assert o.mod_pow(2, 32, p) == p - 1


def pin_max_length(o):
    facts = {r[0]: r[1:] for r in golden("number_facts.txt")}
    m, top = int(facts["max_len_prime"][0]), int(facts["max_len_log2"][0])
    nmax = o.order(2, m)
    for n in range(top + 1):
        N = 1 << n
        w = o.root(m, N, nmax)
        assert o.mod_pow(w, N, m) == 1
        if N > 1:
            assert o.mod_pow(w, N // 2, m) == m - 1      # primitive: w^(N/2) = -1
    try:
        o.root(m, 1 << (top + 1), nmax)
    except ValueError:
        pass
    else:
        raise AssertionError("length 2^(top+1) accepted")


def pin_inverse(o):
    # closed form for m = 13 * 2^20 + 1: N * (m - (m-1)/N) = N m - (m - 1) = 1 (mod m)
    for n in range(20):
        N = 1 << n
        assert o.mod_inverse(N, M) == M - (M - 1) // N
    # brute force for small moduli
    for m in (5, 7, 17, 641):
        for a in range(1, m):
            want = [b for b in range(m) if (a * b) % m == 1]
            assert o.mod_inverse(a, m) == want[0]
    assert o.mod_inverse(6, 9) is None


def pin_mod_mul(o):
    # brute force by repeated addition on small operands, and the 64-bit word edge
    for m in (7, 16, 641):
        for a in range(0, 3 * m, 5):
            for b in range(0, m, 3):
                s = 0
                for _ in range(b):
                    s = (s + a) % m
                assert o.mod_mul(a, b, m) == s
    # (m-1)^2 = 1 (mod m) for any m, checked at the largest words used
    for m in (M, M64, (1 << 61) - 1):
        assert o.mod_mul(m - 1, m - 1, m) == 1


def pin_hand_example(o):
    d = {r[0]: [int(v) for v in r[1:]] for r in golden("hand_ntt_m5.txt")}
    m, w = d["m"][0], d["w"][0]
    assert list(o.ntt(d["x"], m, w)) == d["X"]
    assert list(o.intt(d["X"], m, w)) == d["x"]
    assert list(o.conv(d["f"], d["g"], m)) == d["h"]


def pin_impulses(o):
    # Eq. 2 of an impulse at k is X(u) = w^(uk): fixes the sign and the index
    # of the exponent; together with linearity it fixes the whole map.
    for m, nmax in SMALL[:3]:
        for N in (2, 4, 8, 16):
            if nmax % N:
                continue
            w = o.root(m, N, nmax)
            for k in range(N):
                x = np.zeros(N, dtype=np.uint64)
                x[k] = 1
                X = o.ntt(x, m, w)
                assert [int(v) for v in X] == [o.mod_pow(w, u * k, m) for u in range(N)]


def pin_constant(o):
    for m, nmax in SMALL:
        N = min(64, nmax)
        w = o.root(m, N, nmax)
        c = m - 3
        X = o.ntt(np.full(N, c, dtype=np.uint64), m, w)
        assert int(X[0]) == (N * c) % m and not X[1:].any()


def pin_roundtrip_linear(o):
    r = _rng(1)
    for m, nmax in SMALL + [(M64, 1 << 20)]:
        for N in (1, 2, 8, 64, 256):
            if nmax % N:
                continue
            w = o.root(m, N, nmax)
            x = r.integers(0, m, N, dtype=np.uint64)
            y = r.integers(0, m, N, dtype=np.uint64)
            X, Y = o.ntt(x, m, w), o.ntt(y, m, w)
            assert np.array_equal(o.intt(X, m, w), x)
            a, b = int(r.integers(1, m)), int(r.integers(1, m))
            z = np.array([(a * int(p) + b * int(q)) % m for p, q in zip(x, y)], dtype=np.uint64)
            Z = o.ntt(z, m, w)
            assert [int(v) for v in Z] == [(a * int(p) + b * int(q)) % m for p, q in zip(X, Y)]
            assert int(X[0]) == sum(int(v) for v in x) % m


def pin_conv_closed_forms(o):
    r = _rng(2)
    for m, _ in SMALL:
        for N in (1, 4, 16):
            g = r.integers(0, m, N, dtype=np.uint64)
            for k in range(N):
                d = np.zeros(N, dtype=np.uint64)
                d[k] = 1
                assert np.array_equal(o.conv(d, g, m), np.roll(g, k))   # delta_k * g = shift by k
            f = r.integers(0, m, N, dtype=np.uint64)
            c = int(r.integers(0, m))
            h = o.conv(f, np.full(N, c, dtype=np.uint64), m)
            assert all(int(v) == (c * sum(int(t) for t in f)) % m for v in h)


def pin_theorem(o):
    r = _rng(3)
    for m, nmax in SMALL + [(M64, 1 << 20)]:
        for N in (2, 4, 32, 128):
            if nmax % N:
                continue
            w = o.root(m, N, nmax)
            f = r.integers(0, m, N, dtype=np.uint64)
            g = r.integers(0, m, N, dtype=np.uint64)
            assert np.array_equal(o.ntt_conv(f, g, m, w), o.conv(f, g, m))


def pin_exhaustive_small(o):
    # every length-2 and length-4 input mod 17 (root 2^(8/N)) round-trips, and
    # every length-2 pair convolves as the theorem says
    m, nmax = 17, 8
    for N in (2, 4):
        w = o.root(m, N, nmax)
        grids = np.stack(np.meshgrid(*[np.arange(m, dtype=np.uint64)] * N, indexing="ij"), -1).reshape(-1, N)
        step = 1 if N == 2 else 7
        for x in grids[::step]:
            assert np.array_equal(o.intt(o.ntt(x, m, w), m, w), x)
    w = o.root(m, 2, nmax)
    for f0 in range(m):
        for f1 in range(0, m, 4):
            f = np.array([f0, f1], dtype=np.uint64)
            g = np.array([f1, (f0 + 3) % m], dtype=np.uint64)
            assert np.array_equal(o.ntt_conv(f, g, m, w), o.conv(f, g, m))


def pin_fast_matches_direct(o):
    r = _rng(4)
    for m, nmax in SMALL + [(M64, 1 << 20)]:
        for N in (1, 2, 16, 64, 512):
            if nmax % N:
                continue
            w = o.root(m, N, nmax)
            f = r.integers(0, m, N, dtype=np.uint64)
            g = r.integers(0, m, N, dtype=np.uint64)
            assert np.array_equal(o.fast_conv(f, g, m, w), o.conv(f, g, m))
            assert np.array_equal(o.fast_ntt(f, m, w), o.ntt(f, m, w))


def pin_conv_sample(o):
    # The sampler evaluates Eq. 1 at a list of output indices (read modulo N,
    # the circular index of reading R5).  Three independent anchors:
    #  - an impulse at k: h(j) = g(<j - k>_N) in closed form;
    #  - the full direct convolution, itself pinned above, at the same indices;
    #  - the radix-2 convolution (a different algorithm) at a length where the
    #    full direct one is slow.
    # The index lists are repeated, out of order and past N, so a sampler
    # that reads the list position, drops the reduction or shifts an index fails.
    r = _rng(6)
    for m, nmax in [(641, 64), (2424833, 1024), (M, 1 << 19), (M64, 1 << 20)]:
        N = min(64, nmax)
        g = r.integers(0, m, N, dtype=np.uint64)
        idx = np.array([N - 1, 0, 5, 5, 2 * N + 3, N, 17 % N, 1], dtype=np.uint64)
        for k in (0, 1, N - 1, 9 % N):
            d = np.zeros(N, dtype=np.uint64)
            d[k] = 1
            got = o.conv_sample(d, g, m, idx)
            assert [int(v) for v in got] == [int(g[(int(j) - k) % N]) for j in idx]
        f = r.integers(0, m, N, dtype=np.uint64)
        full = o.conv(f, g, m)
        perm = np.concatenate([r.permutation(N), r.integers(0, 4 * N, 16)]).astype(np.uint64)
        got = o.conv_sample(f, g, m, perm)
        assert [int(v) for v in got] == [int(full[int(j) % N]) for j in perm]
    m, nmax, N = M, 1 << 19, 1 << 12
    w = o.root(m, N, nmax)
    f = r.integers(0, m, N, dtype=np.uint64)
    g = r.integers(0, m, N, dtype=np.uint64)
    fast = o.fast_conv(f, g, m, w)
    idx = r.integers(0, 3 * N, 64).astype(np.uint64)
    assert [int(v) for v in o.conv_sample(f, g, m, idx)] == [int(fast[int(j) % N]) for j in idx]
    assert o.conv_sample(f, g, m, np.zeros(0, dtype=np.uint64)).shape == (0,)


def pin_prime64(o):
    assert M64 == 33629 * (1 << 21) + 1           # Euler form k * 2^(n+2) + 1, n = 19
    assert o.is_prime(M64)
    assert o.mod_pow(2, 1 << 19, M64) == M64 - 1  # M64 | F_19
    assert o.order(2, M64, 1 << 21) == 1 << 20


PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]


def run_pins(o, pins=None):
    failed = []
    for fn in pins or PINS:
        try:
            fn(o)
        except Exception as exc:                  # noqa: BLE001 - any failure counts
            failed.append(f"{fn.__name__}: {type(exc).__name__}: {exc}"[:200])
    return failed
