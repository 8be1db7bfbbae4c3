// ntt_shift.cu -- the strict bit-shift form of the transform (Sec. I, Eq. 2
// and 3 "only bit-shifting, modulo and addition"; Sec. III-A, Prop. 2) for
// the regime where it is literal: a Rader prime m dividing a Fermat number
// F_t = 2^(2^t) + 1 with ord_m(2) = 2^(t+1), so every twiddle is 2^e with
// e < 2^t and N <= 2^(t+1) (t = 4: m = 65537, N <= 32; t = 5: m = 641 or
// 6700417, N <= 64).
//
// SHIFT mode computes the convolution modulo F_t (a multiple of m) and
// reduces modulo m at the end:
//   * a twiddle product b 2^e (b <= 2^(2^t), e < 2^t) is the shift b << e
//     followed by the reduction lo - hi modulo F_t (2^(2^t) = -1): no
//     multiply in any butterfly;
//   * N^-1 = 2^-L = -2^(2^t - L) modulo F_t is a shift and a negation;
//   * the N pointwise products F G are genuine products (the convolution
//     theorem needs them), reduced the same way;
//   * the final residue modulo m uses one Shoup product per output.
// SHOUP mode is the same kernel with every twiddle applied as a Shoup
// product modulo m (the multiply form of the main path), for comparison.
//
// Layout: P = min(32, N) lanes per pair, E = N / P (1 or 2) elements per
// lane, element x = q + P k (q = lane in the group).  Butterflies at a
// distance below P exchange values with __shfl_xor_sync; at distance P
// (N = 64) they are inside the lane.  Forward: the node tree of the main
// path (node i = x >> (L - d), twiddle w^brv(i)); inverse: its transpose
// (Gentleman-Sande butterflies, same twiddles), output at <-x>_N.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/ntt_gb300.h"
#include "ntt_count.h"
#include "ntt_internal.h"
#include "nt_host.h"

namespace {

constexpr int BLK = 256;

struct ShiftArgs {
    const uint32_t *f;
    const uint32_t *g;
    uint32_t *h;
    long long batch;
    uint64_t m;              // the Rader prime (result modulus)
    uint64_t onep;           // floor(2^64 / m)
    // SHOUP mode: twiddles z_i = w^brv(i) mod m and Shoup quotients, i < N/2
    uint32_t z[32];
    uint32_t zp[32];
    uint32_t ninv, ninvp;    // N^-1 mod m, Shoup quotient (SHOUP mode)
};

// ---- arithmetic modulo F_t = 2^K + 1, K = 2^t, values in [0, 2^K] ----
template <int K>
__device__ __forceinline__ uint64_t f_reduce(uint64_t y)     // y < 2^(2K): y = hi 2^K + lo = lo - hi
{
    constexpr uint64_t F = (1ull << K) + 1;
    const uint64_t lo = y & ((1ull << K) - 1), hi = y >> K;
    return lo >= hi ? lo - hi : lo + F - hi;
}
template <int K>
__device__ __forceinline__ uint64_t f_add(uint64_t a, uint64_t b)
{
    constexpr uint64_t F = (1ull << K) + 1;
    const uint64_t s = a + b;
    return s >= F ? s - F : s;
}
template <int K>
__device__ __forceinline__ uint64_t f_sub(uint64_t a, uint64_t b)
{
    constexpr uint64_t F = (1ull << K) + 1;
    return a >= b ? a - b : a + F - b;
}
template <int K>
__device__ __forceinline__ uint64_t f_shl(uint64_t b, uint32_t e)  // b 2^e, e < K, b <= 2^K: b << e < 2^(2K)
{
    return f_reduce<K>(b << e);
}
template <int K>
__device__ __forceinline__ uint64_t f_mul(uint64_t a, uint64_t b)  // general product (pointwise only)
{
    constexpr uint64_t F = (1ull << K) + 1;
    if (a == (1ull << K)) return b == 0 ? 0 : F - b;               // 2^K = -1
    if (b == (1ull << K)) return a == 0 ? 0 : F - a;
    return f_reduce<K>(a * b);                                      // a, b < 2^K: a b < 2^(2K)
}

// ---- arithmetic modulo m (SHOUP mode), canonical values ----
__device__ __forceinline__ uint32_t m_shoup(uint32_t b, uint32_t z, uint32_t zp, uint32_t m)
{
    uint32_t r = b * z - __umulhi(b, zp) * m;
    return r >= m ? r - m : r;
}

// Exponent of the twiddle of node i at length 2^L: w = 2^(2K/N), z_i = w^brv_{L-1}(i).
template <int K, int L>
__device__ __forceinline__ uint32_t tw_exp(uint32_t i)
{
    return (2u * K >> L) * (__brev(i) >> (32 - (L - 1 > 0 ? L - 1 : 1))) * (L > 1 ? 1u : 0u);
}

template <int K, int L, bool SHIFT>
struct Ops {
    using V = uint64_t;
    __device__ static V tw(V b, uint32_t node, const ShiftArgs &a)
    {
        if constexpr (SHIFT) return f_shl<K>(b, tw_exp<K, L>(node));
        else return m_shoup((uint32_t)b, a.z[node], a.zp[node], (uint32_t)a.m);
    }
    __device__ static V add(V x, V y, const ShiftArgs &a)
    {
        if constexpr (SHIFT) return f_add<K>(x, y);
        else { const uint64_t s = x + y; return s >= a.m ? s - a.m : s; }
    }
    __device__ static V sub(V x, V y, const ShiftArgs &a)
    {
        if constexpr (SHIFT) return f_sub<K>(x, y);
        else return x >= y ? x - y : x + a.m - y;
    }
};

template <int K, int L, bool SHIFT>
__global__ void __launch_bounds__(BLK) k_conv_shift(const __grid_constant__ ShiftArgs a)
{
    constexpr int N = 1 << L, P = N < 32 ? N : 32, E = N / P;
    static_assert(E == 1 || E == 2, "N <= 64");
    using O = Ops<K, L, SHIFT>;
    const int lane = threadIdx.x & 31;
    const uint32_t q = (uint32_t)(lane & (P - 1));
    const unsigned FULL = 0xffffffffu;
    const long long gwarp = ((long long)blockIdx.x * BLK + threadIdx.x) >> 5;
    const long long nwarp = ((long long)gridDim.x * BLK) >> 5;
    constexpr int PPW = 32 / P;                         // pairs per warp
    for (long long base = gwarp * PPW; base < a.batch; base += nwarp * PPW) {
        const long long pair = base + lane / P;
        const bool live = pair < a.batch;
        uint64_t v[2][E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const uint32_t x = q + (uint32_t)(P * k);
            v[0][k] = live ? a.f[pair * N + x] : 0;
            v[1][k] = live ? a.g[pair * N + x] : 0;
        }
        // forward node tree, levels d = 0 .. L-1 (distance D = 2^(L-1-d))
#pragma unroll
        for (int d = 0; d < L; ++d) {
            const int D = 1 << (L - 1 - d);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (D >= P) {                               // inside the lane: elements k = 0 (a), 1 (b)
                    const uint64_t t = O::tw(v[s][1], 0u, a);   // node (q + P k) >> (L - d) = 0 at d = 0
                    const uint64_t x0 = v[s][0];
                    v[s][0] = O::add(x0, t, a);
                    v[s][1] = O::sub(x0, t, a);
                } else {
#pragma unroll
                    for (int k = 0; k < E; ++k) {
                        const uint32_t x = q + (uint32_t)(P * k);
                        const uint32_t node = x >> (L - d);
                        const uint64_t mine = v[s][k];
                        const uint64_t other = __shfl_xor_sync(FULL, mine, D);
                        v[s][k] = (q & D) ? O::sub(other, O::tw(mine, node, a), a)
                                          : O::add(mine, O::tw(other, node, a), a);
                    }
                }
            }
        }
        // pointwise product with N^-1
#pragma unroll
        for (int k = 0; k < E; ++k) {
            if constexpr (SHIFT) {
                const uint64_t p = f_mul<K>(v[0][k], v[1][k]);
                const uint64_t t = f_shl<K>(p, (uint32_t)(K - L));   // 2^(K - L) = -2^-L
                v[0][k] = t == 0 ? 0 : (1ull << K) + 1 - t;
            } else {
                const uint32_t m = (uint32_t)a.m;
                const uint64_t p = (v[0][k] * v[1][k]) % m;           // operands < m < 2^24
                v[0][k] = m_shoup((uint32_t)p, a.ninv, a.ninvp, m);
            }
        }
        // inverse: transposed tree, levels d = L-1 .. 0
#pragma unroll
        for (int d = L - 1; d >= 0; --d) {
            const int D = 1 << (L - 1 - d);
            if (D >= P) {
                const uint64_t x0 = v[0][0], x1 = v[0][1];
                v[0][0] = O::add(x0, x1, a);
                v[0][1] = O::tw(O::sub(x0, x1, a), 0u, a);
            } else {
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const uint32_t x = q + (uint32_t)(P * k);
                    const uint32_t node = x >> (L - d);
                    const uint64_t mine = v[0][k];
                    const uint64_t other = __shfl_xor_sync(FULL, mine, D);
                    v[0][k] = (q & D) ? O::tw(O::sub(other, mine, a), node, a) : O::add(mine, other, a);
                }
            }
        }
        // output index <-x>_N, residue modulo m
        if (live) {
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const uint32_t x = q + (uint32_t)(P * k);
                uint64_t r = v[0][k];
                if constexpr (SHIFT) {
                    r = r - __umul64hi(r, a.onep) * a.m;             // r <= 2^K < 2^64: Shoup by 1
                    if (r >= a.m) r -= a.m;
                }
                a.h[pair * N + ((N - x) & (N - 1))] = (uint32_t)r;
            }
        }
    }
}

template <int K, bool SHIFT>
cudaError_t launch(int L, const ShiftArgs &a, int grid, cudaStream_t st)
{
    switch (L) {
#define C(X) case X: if constexpr ((2 * K >> X) >= 1) { k_conv_shift<K, X, SHIFT><<<grid, BLK, 0, st>>>(a); return ntt::launched(); } break;
    C(1) C(2) C(3) C(4) C(5) C(6)
#undef C
    default: break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

extern "C" ntt_status conv_circular_shift(uint64_t m, uint32_t N, const uint32_t *f, const uint32_t *g, uint32_t *h,
                                          size_t batch, int mode, ntt_stream_t stream)
{
    if (!f || !g || !h || batch == 0 || (mode != NTT_SHIFT_STRICT && mode != NTT_SHIFT_SHOUP))
        return ntt_fail(NTT_ERR_ARG, "conv_circular_shift: invalid argument");
    int t = 0;
    if (m > 2 && ((1ull << 32) + 1) % m == 0) t = 5;
    else if (m > 2 && ((1ull << 16) + 1) % m == 0) t = 4;
    if (t == 0 || !nt::is_prime(m))
        return ntt_fail(NTT_ERR_MODULUS, "conv_circular_shift: m=%llu is not a prime factor of F_4 or F_5",
                        (unsigned long long)m);
    const uint32_t nmax = 2u << t;                       // ord_m(2) = 2^(t+1)
    if (nt::order_of_two_pow2(m) != nmax)
        return ntt_fail(NTT_ERR_MODULUS, "conv_circular_shift: ord_m(2) != 2^%d", t + 1);
    if (N < 2 || (N & (N - 1)) || N > nmax)
        return ntt_fail(NTT_ERR_LENGTH, "conv_circular_shift: N=%u must be a power of two in 2..%u", N, nmax);
    int L = 0;
    while ((1u << L) < N) ++L;
    ShiftArgs a{};
    a.f = f; a.g = g; a.h = h; a.batch = (long long)batch; a.m = m;
    a.onep = (uint64_t)(((unsigned __int128)1 << 64) / m);
    const uint64_t w = nt::pow_mod(2, nmax / N, m);
    for (uint32_t i = 0; i < N / 2; ++i) {
        uint32_t r = 0;
        for (int k = 0; k < L - 1; ++k) r |= ((i >> k) & 1u) << (L - 2 - k);
        a.z[i] = (uint32_t)nt::pow_mod(w, r, m);
        a.zp[i] = (uint32_t)(((uint64_t)a.z[i] << 32) / m);
    }
    a.ninv = (uint32_t)nt::pow_mod(N % m, m - 2, m);
    a.ninvp = (uint32_t)(((uint64_t)a.ninv << 32) / m);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long pairs_per_block = (long long)(BLK / 32) * (32 / (N < 32 ? N : 32));
    const long long need = ((long long)batch + pairs_per_block - 1) / pairs_per_block;
    const int grid = (int)(need < (long long)nsm * 8 ? need : (long long)nsm * 8);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (t == 5) e = mode == NTT_SHIFT_STRICT ? launch<32, true>(L, a, grid, st) : launch<32, false>(L, a, grid, st);
    else e = mode == NTT_SHIFT_STRICT ? launch<16, true>(L, a, grid, st) : launch<16, false>(L, a, grid, st);
    if (e != cudaSuccess) return ntt_fail(NTT_ERR_CUDA, "conv_circular_shift: %s", cudaGetErrorString(e));
    return NTT_OK;
}
