// nt_host.h -- host number theory for plan construction (Sec. I, Sec. II,
// Sec. III-A, Appendix A/B of the paper).  Independent of the test oracle:
// primality by deterministic Miller-Rabin, the order of 2 by repeated
// squaring, inverses by Fermat's little theorem.
#pragma once

#include <cstdint>
#include <vector>

namespace nt {

typedef unsigned __int128 u128;

inline uint64_t mul_mod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

inline uint64_t pow_mod(uint64_t a, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mul_mod(r, a, m);
        a = mul_mod(a, a, m);
        e >>= 1;
    }
    return r;
}

// Deterministic Miller-Rabin for n < 2^64 (first twelve prime bases).
inline bool is_prime(uint64_t n)
{
    if (n < 2) return false;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t p : small) {
        if (n == p) return true;
        if (n % p == 0) return false;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (uint64_t a : small) {
        uint64_t x = pow_mod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = mul_mod(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

// ord_m(2) when it is a power of two (2 a lambda-root of order 2^k, Prop. 2),
// else 0: square 2, 2^2, 2^4, ... until the value 1 appears.
inline uint64_t order_of_two_pow2(uint64_t m)
{
    uint64_t x = 2 % m;
    for (int k = 0; k < 63; ++k) {
        if (x == 1) return 1ull << k;
        x = mul_mod(x, x, m);
    }
    return 0;
}

// m^{-1} mod 2^B for odd m (Newton iteration), B = 32 or 64.
inline uint64_t inv_pow2(uint64_t m, int B)
{
    uint64_t x = m;                       // correct to 3 bits
    for (int i = 0; i < 6; ++i) x *= 2 - m * x;
    return B == 32 ? (x & 0xffffffffull) : x;
}

// (x 2^B) mod m
inline uint64_t shl_mod(uint64_t x, int B, uint64_t m) { return (uint64_t)(((u128)x << B) % m); }

// Shoup's quotient floor(z 2^B / m) for z < m
inline uint64_t shoup_quot(uint64_t z, uint64_t m, int B) { return (uint64_t)(((u128)z << B) / m); }

// 2^k mod m for k = 0 .. count-1, by doubling: shift left, subtract m once.
inline std::vector<uint64_t> powers_of_two_by_doubling(uint64_t count, uint64_t m)
{
    std::vector<uint64_t> p(count ? count : 1);
    uint64_t v = 1 % m;
    for (uint64_t k = 0; k < count; ++k) {
        p[k] = v;
        v <<= 1;
        if (v >= m) v -= m;
    }
    return p;
}

inline uint64_t bit_reverse(uint64_t i, int bits)
{
    uint64_t r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1ull) << (bits - 1 - b);
    return r;
}

}  // namespace nt
