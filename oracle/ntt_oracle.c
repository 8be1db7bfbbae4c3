/*
 * Test oracle for the exact digital circular convolution of Chandra,
 * "Fast Digital Convolutions using Bit-Shifts" (arXiv 1005.1497).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Everything here is the plain definition, written out slowly:
 *   - residues  <a>_m with 0 <= <a>_m < m                (Appendix A, Sino notation)
 *   - products through unsigned __int128, so any m < 2^63 is exact
 *   - modular exponentiation by square-and-multiply       (Sec. I, "logarithmic complexity")
 *   - multiplicative inverse by the extended Euclidean algorithm (Appendix A)
 *   - primality by trial division                          (plain definition)
 *   - multiplicative order: smallest nu >= 1 with a^nu = 1 (Eq. LambdaRoot, Sec. II)
 *   - forward transform  X(u) = < sum_t <x(t) w^{ut}>_m >_m          (Eq. 2)
 *   - inverse transform  x(t) = < N^-1 sum_u <X(u) w^{-ut}>_m >_m    (Eq. 3)
 *   - circular convolution h(j) = < sum_k f(k) g(<j-k>_N) >_m       (Eq. 1)
 *   - a textbook radix-2 Cooley-Tukey convolution, with e^{2 pi i a/N}
 *     replaced by powers of the integer root (Sec. I), for lengths where
 *     the O(N^2) definitions are too slow; it is pinned against them.
 *   - the exact integer circular convolution (Eq. 1 with no modulus),
 *     accumulated in signed __int128
 *   - the modulus-free transform and convolution modulo 2^alpha (Sec. III-B)
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   R1  Eq. 2 reduces each term; the sum is reduced too, so X(u) is canonical.
 *   R2  For N < N_Max the kernel 2^{ut} is read as w^{ut} with w = 2^{N_Max/N}
 *       (Sec. I: lengths N = 2^n that divide N_Max).  w is still a power of two.
 *   R3  2^{-ut} is read as w^{<-ut>_N}; the printed 2^{N-ut} holds only for ut < N.
 *   R5  g(j-k) in Eq. 1 is read circularly, g(<j-k>_N).
 *
 * Mutation hooks (ORACLE_MUTANT) exist only so that a test can build
 * deliberately wrong copies of this oracle and prove that the pins reject
 * them.  The default build defines none of them.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

typedef unsigned __int128 u128;

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* <a * b>_m  (Appendix A) */
uint64_t or_mod_mul(uint64_t a, uint64_t b, uint64_t m)
{
    return (uint64_t)(((u128)a * (u128)b) % (u128)m);
}

/* <a + b>_m for a, b < m */
static uint64_t mod_add(uint64_t a, uint64_t b, uint64_t m)
{
    return (uint64_t)(((u128)a + (u128)b) % (u128)m);
}

/* <a^e>_m by square-and-multiply: O(log e) products (Sec. I). */
uint64_t or_mod_pow(uint64_t a, uint64_t e, uint64_t m)
{
    uint64_t result = 1 % m;
    uint64_t base = a % m;
    while (e > 0) {
        if (e & 1u)
            result = or_mod_mul(result, base, m);
        base = or_mod_mul(base, base, m);
        e >>= 1;
    }
    return result;
}

/* Extended Euclid (Appendix A): returns 1 and sets *inv with <a * inv>_m = 1
 * when gcd(a, m) = 1, else returns 0.  Works on signed 128-bit Bezout
 * coefficients so no intermediate overflows for m < 2^63. */
int or_mod_inverse(uint64_t a, uint64_t m, uint64_t *inv)
{
    __int128 r0 = (__int128)m, r1 = (__int128)(a % m);
    __int128 s0 = 0, s1 = 1;           /* coefficients of a */
    while (r1 != 0) {
        __int128 q = r0 / r1;
        __int128 r2 = r0 - q * r1;
        __int128 s2 = s0 - q * s1;
        r0 = r1; r1 = r2;
        s0 = s1; s1 = s2;
    }
    if (r0 != 1)
        return 0;
    __int128 v = s0 % (__int128)m;
    if (v < 0)
        v += (__int128)m;
    *inv = (uint64_t)v;
    return 1;
}

/* Primality by trial division over every candidate divisor d with d*d <= m. */
int or_is_prime(uint64_t m)
{
    if (m < 2)
        return 0;
    if (m < 4)
        return 1;
    if (m % 2 == 0)
        return 0;
    for (uint64_t d = 3; (u128)d * d <= m; d += 2)
        if (m % d == 0)
            return 0;
    return 1;
}

/* Multiplicative order (Eq. LambdaRoot): the smallest nu >= 1 with
 * <a^nu>_m = 1, found by walking the successive powers a, a^2, ... (the
 * "digital circle" of Fig. 1).  Returns 0 when no such nu <= limit exists
 * (including gcd(a, m) != 1). */
uint64_t or_order(uint64_t a, uint64_t m, uint64_t limit)
{
    if (m == 1)
        return 1;
    uint64_t p = a % m;
    for (uint64_t nu = 1; nu <= limit; nu++) {
        if (p == 1)
            return nu;
        p = or_mod_mul(p, a, m);
    }
    return 0;
}

/* Successive powers w^0 .. w^{count-1} mod m (the harmonics of Eq. 2). */
static uint64_t *powers(uint64_t w, uint64_t count, uint64_t m)
{
    uint64_t *pw = (uint64_t *)malloc(sizeof(uint64_t) * (count ? count : 1));
    if (!pw)
        return NULL;
    uint64_t p = 1 % m;
    for (uint64_t k = 0; k < count; k++) {
        pw[k] = p;
        p = or_mod_mul(p, w, m);
    }
    return pw;
}

/* Eq. 2, direct O(N^2): X(u) = < sum_t <x(t) * w^{<ut>_N}>_m >_m.
 * w must have order N (w^N = 1).  Returns 0 on success. */
int or_ntt(const uint64_t *x, uint64_t *X, uint64_t N, uint64_t m, uint64_t w)
{
    uint64_t *pw = powers(w, N, m);
    if (!pw)
        return -1;
    for (uint64_t u = 0; u < N; u++) {
        uint64_t acc = 0;
        for (uint64_t t = 0; t < N; t++) {
#if ORACLE_MUTANT == 2
            uint64_t e = (uint64_t)(((u128)(N - u % N) * t) % N);   /* wrong sign */
#else
            uint64_t e = (uint64_t)(((u128)u * t) % N);
#endif
            acc = mod_add(acc, or_mod_mul(x[t] % m, pw[e], m), m);
        }
        X[u] = acc;
    }
    free(pw);
    return 0;
}

/* Eq. 3, direct O(N^2): x(t) = < N^-1 * sum_u <X(u) * w^{<-ut>_N}>_m >_m,
 * with N^-1 from the extended Euclidean algorithm (Appendix A). */
int or_intt(const uint64_t *X, uint64_t *x, uint64_t N, uint64_t m, uint64_t w)
{
    uint64_t ninv;
    if (!or_mod_inverse(N % m, m, &ninv))
        return -2;
#if ORACLE_MUTANT == 3
    ninv = 1;                                                   /* dropped 1/N */
#endif
    uint64_t *pw = powers(w, N, m);
    if (!pw)
        return -1;
    for (uint64_t t = 0; t < N; t++) {
        uint64_t acc = 0;
        for (uint64_t u = 0; u < N; u++) {
            uint64_t ut = (uint64_t)(((u128)u * t) % N);
#if ORACLE_MUTANT == 4
            uint64_t e = ut;                                    /* root not inverted */
#else
            uint64_t e = (N - ut) % N;                          /* <-ut>_N */
#endif
            acc = mod_add(acc, or_mod_mul(X[u] % m, pw[e], m), m);
        }
        x[t] = or_mod_mul(acc, ninv, m);
    }
    free(pw);
    return 0;
}

/* Eq. 1 at one output index j: < sum_k f(k) g(<j-k>_N) >_m. */
uint64_t or_conv_at(const uint64_t *f, const uint64_t *g, uint64_t N, uint64_t m, uint64_t j)
{
    uint64_t acc = 0;
    for (uint64_t k = 0; k < N; k++) {
#if ORACLE_MUTANT == 1
        uint64_t idx = (j + k) % N;                             /* wrong index sign */
#elif ORACLE_MUTANT == 5
        uint64_t idx = (j + N - k) % N;
        if (k == N - 1) break;                                  /* dropped term */
#else
        uint64_t idx = (j + N - k % N) % N;
#endif
        acc = mod_add(acc, or_mod_mul(f[k] % m, g[idx] % m, m), m);
    }
    return acc;
}

/* Eq. 1, direct O(N^2) over every output index. */
void or_conv(const uint64_t *f, const uint64_t *g, uint64_t *h, uint64_t N, uint64_t m)
{
    for (uint64_t j = 0; j < N; j++)
        h[j] = or_conv_at(f, g, N, m, j);
}

/* Eq. 1 at a list of output indices (sampled parity at large N). */
void or_conv_sample(const uint64_t *f, const uint64_t *g, uint64_t N, uint64_t m,
                    const uint64_t *idx, uint64_t count, uint64_t *out)
{
    for (uint64_t i = 0; i < count; i++) {
#if ORACLE_MUTANT == 8
        out[i] = or_conv_at(f, g, N, m, i % N);                 /* list position, not the index */
#elif ORACLE_MUTANT == 9
        out[i] = or_conv_at(f, g, N, m, (idx[i] + 1) % N);      /* off by one output */
#else
        out[i] = or_conv_at(f, g, N, m, idx[i] % N);
#endif
    }
}

/* The convolution theorem with the direct transforms: Eq. 2 on f and g, the
 * pointwise product <F(u) G(u)>_m, then Eq. 3.  O(N^2). */
int or_ntt_conv(const uint64_t *f, const uint64_t *g, uint64_t *h, uint64_t N, uint64_t m, uint64_t w)
{
    uint64_t *F = (uint64_t *)malloc(sizeof(uint64_t) * N);
    uint64_t *G = (uint64_t *)malloc(sizeof(uint64_t) * N);
    if (!F || !G) { free(F); free(G); return -1; }
    int rc = or_ntt(f, F, N, m, w);
    if (!rc) rc = or_ntt(g, G, N, m, w);
    if (!rc) {
        for (uint64_t u = 0; u < N; u++)
            F[u] = or_mod_mul(F[u], G[u], m);
        rc = or_intt(F, h, N, m, w);
    }
    free(F); free(G);
    return rc;
}

/* Textbook iterative radix-2 Cooley-Tukey transform (Sec. I: replace
 * e^{2 pi i a/N} by the powers of the integer root w of order N):
 * bit-reversal permutation, then butterflies (a, b) -> (a + w^j b, a - w^j b)
 * over half-lengths 1, 2, 4, ..., N/2.  Natural order in and out. */
static void radix2_transform(uint64_t *a, uint64_t N, uint64_t m, uint64_t w)
{
    for (uint64_t i = 1, j = 0; i < N; i++) {
        uint64_t bit = N >> 1;
        for (; j & bit; bit >>= 1)
            j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (uint64_t len = 2; len <= N; len <<= 1) {
        uint64_t wlen = or_mod_pow(w, N / len, m);   /* root of order len */
        for (uint64_t s = 0; s < N; s += len) {
            uint64_t wj = 1 % m;
            for (uint64_t j = 0; j < len / 2; j++) {
                uint64_t u = a[s + j];
                uint64_t v = or_mod_mul(a[s + j + len / 2], wj, m);
                a[s + j] = mod_add(u, v, m);
                a[s + j + len / 2] = mod_add(u, m - v, m);
                wj = or_mod_mul(wj, wlen, m);
            }
        }
    }
}

/* Fast radix-2 convolution: forward transforms of f and g with w, pointwise
 * product, forward transform with w^-1, scaling by N^-1.  N a power of two. */
int or_fast_conv(const uint64_t *f, const uint64_t *g, uint64_t *h, uint64_t N, uint64_t m, uint64_t w)
{
    uint64_t winv, ninv;
    if (!or_mod_inverse(w, m, &winv) || !or_mod_inverse(N % m, m, &ninv))
        return -2;
    uint64_t *F = (uint64_t *)malloc(sizeof(uint64_t) * N);
    uint64_t *G = (uint64_t *)malloc(sizeof(uint64_t) * N);
    if (!F || !G) { free(F); free(G); return -1; }
    for (uint64_t i = 0; i < N; i++) { F[i] = f[i] % m; G[i] = g[i] % m; }
    radix2_transform(F, N, m, w);
    radix2_transform(G, N, m, w);
    for (uint64_t i = 0; i < N; i++)
        F[i] = or_mod_mul(F[i], G[i], m);
    radix2_transform(F, N, m, winv);
    for (uint64_t i = 0; i < N; i++)
        h[i] = or_mod_mul(F[i], ninv, m);
    free(F); free(G);
    return 0;
}

/* Forward transform by the radix-2 algorithm (natural order), for large-N
 * checks of the spectrum. */
int or_fast_ntt(const uint64_t *x, uint64_t *X, uint64_t N, uint64_t m, uint64_t w)
{
    for (uint64_t i = 0; i < N; i++)
        X[i] = x[i] % m;
    radix2_transform(X, N, m, w);
    return 0;
}

/* ---- Exact integer circular convolution -------------------------------
 * Eq. 1 without the modulus: h(j) = sum_k f(k) g(<j-k>_N) over the
 * integers, accumulated in signed __int128 (the "exact digital filtering"
 * that Sec. I and the Conclusion aim at; recovering it from residues is the
 * Chinese remainder theorem, which this oracle does not use).  Inputs are
 * signed 64-bit.  Returns 0 when every h(j) fits a signed 64-bit word, -1
 * otherwise (h then holds the low 64 bits). */
typedef __int128 i128;

static int int_conv_at(const int64_t *f, const int64_t *g, uint64_t N, uint64_t j, int64_t *out)
{
    i128 acc = 0;
    for (uint64_t k = 0; k < N; k++) {
#if ORACLE_MUTANT == 6
        uint64_t idx = (j + k) % N;                             /* wrong index sign */
#else
        uint64_t idx = (j + N - k) % N;                         /* <j-k>_N */
#endif
        acc += (i128)f[k] * (i128)g[idx];
    }
    *out = (int64_t)acc;
    return (acc >= -(((i128)1) << 63) && acc < (((i128)1) << 63)) ? 0 : -1;
}

int or_int_conv(const int64_t *f, const int64_t *g, int64_t *h, uint64_t N)
{
    int rc = 0;
    for (uint64_t j = 0; j < N; j++)
        rc |= int_conv_at(f, g, N, j, &h[j]);
    return rc;
}

int or_int_conv_sample(const int64_t *f, const int64_t *g, uint64_t N, const uint64_t *idx, uint64_t count,
                       int64_t *out)
{
    int rc = 0;
    for (uint64_t i = 0; i < count; i++)
        rc |= int_conv_at(f, g, N, idx[i] % N, &out[i]);
    return rc;
}

/* ---- Modulus-free transform (Sec. III-B) --------------------------------
 * For odd a, a^{2^{alpha-2}} = 1 mod 2^alpha (Eq. Dyadic), so powers of a
 * give a length-N kernel modulo 2^alpha with no division: arithmetic wraps
 * at 2^64 and truncation to alpha bits is the residue.  1 <= alpha <= 64.
 *   X(u) = < sum_t x(t) a^{<ut>_N} >_{2^alpha}           (Eq. 2 with m = 2^alpha)
 *   h(j) = < sum_k f(k) g(<j-k>_N) >_{2^alpha}           (Eq. 1 with m = 2^alpha) */
static uint64_t low_bits(uint64_t v, uint64_t alpha)
{
    return alpha >= 64 ? v : (v & ((((uint64_t)1) << alpha) - 1));
}

int or_dyadic_ntt(const uint64_t *x, uint64_t *X, uint64_t N, uint64_t alpha, uint64_t a)
{
    if (alpha < 1 || alpha > 64 || N == 0)
        return -2;
    uint64_t *pw = (uint64_t *)malloc(sizeof(uint64_t) * N);
    if (!pw)
        return -1;
    uint64_t p = 1;
    for (uint64_t k = 0; k < N; k++) {
        pw[k] = low_bits(p, alpha);
        p *= a;                                                 /* wraps at 2^64 */
    }
    for (uint64_t u = 0; u < N; u++) {
        uint64_t acc = 0;
        for (uint64_t t = 0; t < N; t++)
            acc += x[t] * pw[(uint64_t)(((u128)u * t) % N)];
#if ORACLE_MUTANT == 7
        X[u] = acc;                                             /* not truncated to alpha bits */
#else
        X[u] = low_bits(acc, alpha);
#endif
    }
    free(pw);
    return 0;
}

int or_dyadic_conv(const uint64_t *f, const uint64_t *g, uint64_t *h, uint64_t N, uint64_t alpha)
{
    if (alpha < 1 || alpha > 64)
        return -2;
    for (uint64_t j = 0; j < N; j++) {
        uint64_t acc = 0;
        for (uint64_t k = 0; k < N; k++)
            acc += f[k] * g[(j + N - k) % N];
        h[j] = low_bits(acc, alpha);
    }
    return 0;
}
