// ntt_exact.cuh -- arithmetic of the exact (non-modular) convolution shared
// by its elementwise kernels and the fused convolution kernels: residues of
// signed 64-bit integers modulo each prime, and Garner's mixed-radix form of
// the Chinese remainder theorem back to a signed 64-bit integer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ntt_gb300.h"

namespace ntt {

constexpr int XKMAX = NTT_EXACT_MAX_PRIMES;
typedef unsigned __int128 xu128;
typedef __int128 xi128;

// Residue and reconstruction constants of one prime, passed by value.
struct PrimeC {
    uint64_t m;
    uint64_t onep;        // floor(2^64 / m): Shoup quotient of the factor 1
    uint64_t r64;         // 2^64 mod m
    int word;             // 32 or 64
    int pad;
};

struct ExactArgs {
    int k;                          // number of primes
    int vec;                        // 1: every base is 16-byte aligned (four-element path)
    long long n;                    // elements
    PrimeC p[XKMAX];
    uint64_t inv[XKMAX][XKMAX];     // inv[i][j] = m_i^-1 mod m_j (i < j)
    uint64_t invp[XKMAX][XKMAX];    // floor(inv 2^64 / m_j)
    unsigned long long half_lo, half_hi;   // (M - 1) / 2
    unsigned long long M_lo, M_hi;         // M
    // fused convolution kernels: the prime this launch reduces modulo, the
    // earlier primes' residue arrays ([pairs][N], canonical) and, for the
    // last prime, the signed 64-bit output ([pairs][N])
    int j;
    int pad;
    const void *prev[XKMAX];
    long long *h64;
};

__device__ __forceinline__ uint64_t shoup64(uint64_t b, uint64_t z, uint64_t zp, uint64_t m)
{
    return b * z - __umul64hi(b, zp) * m;           // in [0, 2m) for any b < 2^64
}

__device__ __forceinline__ uint64_t csub64(uint64_t v, uint64_t m) { return v >= m ? v - m : v; }

// <x>_m for a signed 64-bit x: reduce its two's-complement bits, then take
// away 2^64 mod m when x is negative.
__device__ __forceinline__ uint64_t residue(long long x, const PrimeC &p)
{
    uint64_t r = csub64(shoup64((uint64_t)x, 1, p.onep, p.m), p.m);
    if (x < 0) r = r >= p.r64 ? r - p.r64 : r + p.m - p.r64;
    return r;
}

// Garner's mixed-radix reconstruction of one output from its residues.
__device__ __forceinline__ long long garner(const ExactArgs &a, const uint64_t (&r)[XKMAX])
{
    const xu128 half = ((xu128)a.half_hi << 64) | a.half_lo;
    const xu128 M = ((xu128)a.M_hi << 64) | a.M_lo;
    uint64_t v[XKMAX];
#pragma unroll
    for (int j = 0; j < XKMAX; ++j) {
        if (j >= a.k) break;
        const PrimeC &pj = a.p[j];
        uint64_t t = r[j];
        // mixed-radix digit: t = (...((r_j - v_0) c_0j - v_1) c_1j ...) mod m_j
#pragma unroll
        for (int q = 0; q < XKMAX; ++q) {
            if (q >= j) break;
            const uint64_t vq = csub64(shoup64(v[q], 1, pj.onep, pj.m), pj.m);     // v_q mod m_j
            const uint64_t d = t >= vq ? t - vq : t + pj.m - vq;
            t = csub64(shoup64(d, a.inv[q][j], a.invp[q][j], pj.m), pj.m);
        }
        v[j] = t;
    }
    // X = v_0 + m_0 (v_1 + m_1 (v_2 + ...)), Horner from the top digit
    xu128 X = 0;
#pragma unroll
    for (int j = XKMAX - 1; j >= 0; --j)
        if (j < a.k) X = X * a.p[j].m + v[j];
    const xi128 s = X > half ? (xi128)X - (xi128)M : (xi128)X;
    return (long long)s;
}

__device__ __forceinline__ uint64_t load_res(const ExactArgs &a, const void *const *res, int j, long long i)
{
    return a.p[j].word == 32 ? (uint64_t) static_cast<const uint32_t *>(res[j])[i] : static_cast<const uint64_t *>(res[j])[i];
}

}  // namespace ntt
