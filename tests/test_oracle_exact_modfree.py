"""Pins of the oracle's exact integer convolution (Eq. 1 with no modulus,
the target of exact digital filtering, Sec. I) and of its modulus-free
transform modulo 2^alpha (Sec. III-B), against brute force in Python
integers, a library routine, closed forms and the paper's identities.

The modulus-free part also settles the question Sec. III-B leaves open:
powers of an odd a give a length-N kernel modulo 2^alpha (Eq. Dyadic), the
forward half of the convolution property holds, but the orthogonality sum
that an inverse needs vanishes for no root of order N >= 4, so no inverse
transform recovers the convolution."""
import numpy as np
import pytest

TABLE1 = [641, 2424833, 319489, 13631489]


def brute_int_conv(f, g):
    N = len(f)
    return [sum(int(f[k]) * int(g[(j - k) % N]) for k in range(N)) for j in range(N)]


def test_int_conv_brute_force(orc):
    rng = np.random.default_rng(5)
    for N in (1, 2, 3, 5, 8, 13, 16):
        for bound in (3, 1 << 20, 1 << 28):
            f = rng.integers(-bound, bound, N, dtype=np.int64)
            g = rng.integers(-bound, bound, N, dtype=np.int64)
            assert orc.int_conv(f, g).tolist() == brute_int_conv(f, g)


def test_int_conv_library_linear_convolution(orc):
    # circular convolution = linear convolution folded modulo N (numpy's
    # direct integer convolution as the library primitive)
    rng = np.random.default_rng(6)
    for N in (64, 200, 256):
        f = rng.integers(-(1 << 20), 1 << 20, N, dtype=np.int64)
        g = rng.integers(-(1 << 20), 1 << 20, N, dtype=np.int64)
        lin = np.convolve(f, g)
        want = lin[:N].copy()
        want[: N - 1] += lin[N:]
        assert np.array_equal(orc.int_conv(f, g), want)


def test_int_conv_closed_forms(orc):
    rng = np.random.default_rng(7)
    N = 97
    g = rng.integers(-(1 << 30), 1 << 30, N, dtype=np.int64)
    for s in (0, 1, 40, 96):
        delta = np.zeros(N, dtype=np.int64)
        delta[s] = 1
        assert np.array_equal(orc.int_conv(delta, g), np.roll(g, s))          # shift
    ones = np.ones(N, dtype=np.int64)
    assert np.all(orc.int_conv(ones, g) == g.sum())                          # constant
    assert np.array_equal(orc.int_conv(g, ones), orc.int_conv(ones, g))      # commutative
    neg = orc.int_conv(-g, ones)
    assert np.array_equal(neg, -orc.int_conv(g, ones))                        # sign


def test_int_conv_extremes_and_overflow(orc):
    big = np.full(2, (1 << 31) - 1, dtype=np.int64)
    assert np.all(orc.int_conv(big, big) == 2 * ((1 << 31) - 1) ** 2)
    worst = np.full(4, 1 << 31, dtype=np.int64)
    with pytest.raises(OverflowError):                                        # 4 * 2^62 = 2^64
        orc.int_conv(worst, worst)
    # exactly -2^63 fits, 2^63 does not
    two = np.array([1 << 31, 1 << 31], dtype=np.int64)
    mtwo = np.array([-(1 << 31), -(1 << 31)], dtype=np.int64)
    assert np.all(orc.int_conv(two, mtwo) == -(1 << 63))
    with pytest.raises(OverflowError):
        orc.int_conv(two, two)


def test_int_conv_reduces_to_the_modular_convolution(orc):
    rng = np.random.default_rng(8)
    for m in TABLE1:
        N = 32
        f = rng.integers(-(1 << 24), 1 << 24, N, dtype=np.int64)
        g = rng.integers(-(1 << 24), 1 << 24, N, dtype=np.int64)
        h = orc.int_conv(f, g)
        fm = np.array([int(v) % m for v in f], dtype=np.uint64)
        gm = np.array([int(v) % m for v in g], dtype=np.uint64)
        assert [int(v) % m for v in h] == orc.conv(fm, gm, m).tolist()


def test_int_conv_sample(orc):
    rng = np.random.default_rng(9)
    N = 300
    f = rng.integers(-1000, 1000, N, dtype=np.int64)
    g = rng.integers(-1000, 1000, N, dtype=np.int64)
    idx = np.array([0, 1, 299, 150, 600], dtype=np.uint64)
    full = orc.int_conv(f, g)
    assert orc.int_conv_sample(f, g, idx).tolist() == [full[int(i) % N] for i in idx]


# ---- modulus-free transform (Sec. III-B) -----------------------------------

def test_dyadic_identity():
    # Eq. Dyadic: a^(2^(alpha-2)) = 1 mod 2^alpha for every odd a (alpha >= 3),
    # and the exponent is the least such power of two for a = 3 and a = 5
    for alpha in range(3, 15):
        M = 1 << alpha
        for a in range(1, M, 2):
            assert pow(a, 1 << (alpha - 2), M) == 1
        for a in (3, 5):
            assert pow(a, 1 << (alpha - 3), M) != 1


def order_mod(a, M):
    x, k = a % M, 1
    while x != 1:
        x, k = x * a % M, k + 1
    return k


def test_dyadic_ntt_brute_force(orc):
    rng = np.random.default_rng(10)
    for alpha in (5, 16, 33, 64):
        M = 1 << alpha
        a = pow(3, 1 << max(0, alpha - 2 - 3), M)      # an element of order 8
        assert order_mod(a, M) == 8
        x = rng.integers(0, 1 << 62, 8, dtype=np.uint64) % np.uint64(M - 1 if alpha < 64 else (1 << 63))
        want = [sum(int(x[t]) * pow(a, u * t, M) for t in range(8)) % M for u in range(8)]
        assert orc.dyadic_ntt(x, alpha, a).tolist() == want


def test_dyadic_conv_brute_force(orc):
    rng = np.random.default_rng(11)
    for alpha in (7, 32, 64):
        M = 1 << alpha
        f = rng.integers(0, 1 << 40, 9, dtype=np.uint64)
        g = rng.integers(0, 1 << 40, 9, dtype=np.uint64)
        want = [v % M for v in brute_int_conv(f, g)]
        assert orc.dyadic_conv(f, g, alpha).tolist() == want


def test_dyadic_forward_convolution_property_holds(orc):
    # T(f (*) g) = T(f) T(g) mod 2^alpha needs only a^N = 1
    rng = np.random.default_rng(12)
    for alpha, N in ((16, 4), (32, 8), (64, 16)):
        M = 1 << alpha
        a = pow(3, (1 << (alpha - 2)) // N, M)
        assert order_mod(a, M) == N
        f = rng.integers(0, M - 1 if alpha < 64 else 1 << 62, N, dtype=np.uint64)
        g = rng.integers(0, M - 1 if alpha < 64 else 1 << 62, N, dtype=np.uint64)
        lhs = orc.dyadic_ntt(orc.dyadic_conv(f, g, alpha), alpha, a)
        F, G = orc.dyadic_ntt(f, alpha, a), orc.dyadic_ntt(g, alpha, a)
        assert lhs.tolist() == [int(p) * int(q) % M for p, q in zip(F, G)]


def test_dyadic_orthogonality_fails_for_every_root_of_order_4_or_more():
    # sum_j a^(jk) must be 0 mod 2^alpha for 0 < k < N for an inverse to exist
    # (with any normalisation).  Only N = 2 (a = -1) passes.
    for alpha in range(3, 12):
        M = 1 << alpha
        for a in range(3, M, 2):
            N = order_mod(a, M)
            ok = all(sum(pow(a, j * k, M) for j in range(N)) % M == 0 for k in range(1, N))
            if N == 2 and a == M - 1:
                assert ok
            elif N >= 4:
                assert not ok, (alpha, a, N)


def test_dyadic_unnormalised_inverse_does_not_recover_the_convolution(orc):
    # With alpha = 64 >= beta + N (8-bit data, N = 8, Sec. III-B's sizing
    # rule), transforming the product spectrum with a^-1 still does not give
    # N h: the orthogonality sums are not N delta.
    rng = np.random.default_rng(13)
    alpha, N = 64, 8
    M = 1 << alpha
    a = pow(3, (1 << (alpha - 2)) // N, M)
    ainv = pow(a, -1, M)
    f = rng.integers(0, 256, N, dtype=np.uint64)
    g = rng.integers(0, 256, N, dtype=np.uint64)
    F, G = orc.dyadic_ntt(f, alpha, a), orc.dyadic_ntt(g, alpha, a)
    H = np.array([int(p) * int(q) % M for p, q in zip(F, G)], dtype=np.uint64)
    back = orc.dyadic_ntt(H, alpha, ainv)
    # the transform index map: back(t) = sum_s h(s) S(s - t) with S the
    # orthogonality sums; it differs from N h(<-t>_N)
    h = orc.dyadic_conv(f, g, alpha)
    want = [(N * int(h[(-t) % N])) % M for t in range(N)]
    assert back.tolist() != want
    # and the failure is exactly the non-vanishing orthogonality sums
    S = [sum(pow(a, j * k, M) for j in range(N)) % M for k in range(N)]
    pred = [sum(int(h[s]) * S[(s + t) % N] for s in range(N)) % M for t in range(N)]
    assert back.tolist() == pred
