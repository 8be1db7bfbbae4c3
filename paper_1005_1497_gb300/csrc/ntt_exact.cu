// ntt_exact.cu -- exact integer circular convolution (Eq. 1 with no
// modulus): the "exact digital filtering" of Sec. I, obtained from the
// modular convolutions of several Rader primes (Sec. III-A, Table 1 and
// other prime factors of Fermat numbers) and the Chinese remainder theorem.
//
//   1. one elementwise pass splits the signed 64-bit inputs into residues
//      modulo every prime of the plan;
//   2. each prime's residues are convolved by the fused modular path
//      (forward transform, pointwise product, inverse, Eq. 1-3);
//   3. one elementwise pass rebuilds each output from its residues by
//      Garner's mixed-radix form of the Chinese remainder theorem and maps
//      it to the signed range (-M/2, M/2], M the product of the primes.
//
// The result is exact whenever every |h(j)| < 2^bound_bits, the bound the
// caller declares; the plan picks primes whose product exceeds 2^(bound+1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/ntt_gb300.h"
#include "ntt_internal.h"
#include "nt_host.h"
#include "ntt_count.h"
#include "ntt_exact.cuh"

namespace {

constexpr int KMAX = NTT_EXACT_MAX_PRIMES;
typedef unsigned __int128 u128;
typedef __int128 i128;
using ntt::ExactArgs;
using ntt::PrimeC;
using ntt::csub64;
using ntt::garner;
using ntt::load_res;
using ntt::residue;
using ntt::shoup64;

// Four elements per thread (16-byte loads and stores), f and g in one
// launch; a scalar loop takes the tail and unaligned bases.
template <int K, typename T>
__device__ __forceinline__ void put_residues(const ExactArgs &a, void *const *out, long long i, const long long (&x)[4])
{
    const PrimeC &p = a.p[K];
    uint64_t r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) r[e] = residue(x[e], p);
    if constexpr (sizeof(T) == 4) {
        reinterpret_cast<uint4 *>(static_cast<uint32_t *>(out[K]) + i)[0] =
            make_uint4((uint32_t)r[0], (uint32_t)r[1], (uint32_t)r[2], (uint32_t)r[3]);
    } else {
        ulonglong2 *q = reinterpret_cast<ulonglong2 *>(static_cast<uint64_t *>(out[K]) + i);
        q[0] = make_ulonglong2(r[0], r[1]);
        q[1] = make_ulonglong2(r[2], r[3]);
    }
}

__device__ __forceinline__ void residues_scalar(const ExactArgs &a, const long long *x, void *const *out, long long i)
{
    const long long v = x[i];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        if (j >= a.k) break;
        const uint64_t r = residue(v, a.p[j]);
        if (a.p[j].word == 32) static_cast<uint32_t *>(out[j])[i] = (uint32_t)r;
        else static_cast<uint64_t *>(out[j])[i] = r;
    }
}

// Every prime below 2^25 (32-bit words, the usual case): a residue is two
// 32-bit Shoup products, one per half of the input's bits, and for one or
// two primes Garner's reconstruction fits 64-bit arithmetic (M < 2^50).
// The residue arrays travel in the kernel parameters.
struct Exact32 {
    int k;
    int pad;
    long long n;                           // elements of this wave
    uint32_t m[KMAX];
    uint32_t c[KMAX], cp[KMAX];            // 2^32 mod m and its Shoup quotient
    uint32_t onep[KMAX];                   // floor(2^32 / m): Shoup quotient of the factor 1
    uint32_t r64[KMAX];                    // 2^64 mod m
    uint32_t inv01, inv01p;                // m_0^-1 mod m_1 and its Shoup quotient (k == 2)
    unsigned long long M, half;            // k <= 2: the product of the primes and (M - 1) / 2
    uint32_t *rf[KMAX], *rg[KMAX];         // residues of f (the convolutions leave h's there) and of g
};

__device__ __forceinline__ uint32_t shoup32(uint32_t b, uint32_t z, uint32_t zp, uint32_t m)
{
    return b * z - __umulhi(b, zp) * m;     // in [0, 2m) for any b < 2^32
}

// <x>_m of a signed 64-bit x: its bits as hi 2^32 + lo, each half reduced by
// a Shoup product (sum below 4m), then 2^64 mod m taken away if x < 0.
__device__ __forceinline__ uint32_t residue32(long long x, const Exact32 &a, int j)
{
    const uint64_t u = (uint64_t)x;
    const uint32_t lo = (uint32_t)u, hi = (uint32_t)(u >> 32), m = a.m[j];
    uint32_t s = shoup32(hi, a.c[j], a.cp[j], m) + shoup32(lo, 1u, a.onep[j], m);
    s = s >= 2 * m ? s - 2 * m : s;
    s = s >= m ? s - m : s;
    if (x < 0) s = s >= a.r64[j] ? s - a.r64[j] : s + m - a.r64[j];
    return s;
}

template <int K>
__global__ void __launch_bounds__(256) k_exact_residues32(const __grid_constant__ Exact32 a,
                                                          const long long *__restrict__ f,
                                                          const long long *__restrict__ g)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long n4 = a.n / 4;                       // bases are 16-byte aligned (checked by the caller)
    for (long long q = tid; q < n4; q += nthr) {
        const longlong2 f0 = __ldcs(reinterpret_cast<const longlong2 *>(f) + 2 * q);
        const longlong2 f1 = __ldcs(reinterpret_cast<const longlong2 *>(f) + 2 * q + 1);
        const longlong2 g0 = __ldcs(reinterpret_cast<const longlong2 *>(g) + 2 * q);
        const longlong2 g1 = __ldcs(reinterpret_cast<const longlong2 *>(g) + 2 * q + 1);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            reinterpret_cast<uint4 *>(a.rf[j])[q] = make_uint4(residue32(f0.x, a, j), residue32(f0.y, a, j),
                                                               residue32(f1.x, a, j), residue32(f1.y, a, j));
            reinterpret_cast<uint4 *>(a.rg[j])[q] = make_uint4(residue32(g0.x, a, j), residue32(g0.y, a, j),
                                                               residue32(g1.x, a, j), residue32(g1.y, a, j));
        }
    }
    for (long long i = 4 * n4 + tid; i < a.n; i += nthr) {
        const long long x = f[i], y = g[i];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            a.rf[j][i] = residue32(x, a, j);
            a.rg[j][i] = residue32(y, a, j);
        }
    }
}

// Garner for one or two 32-bit primes: v_0 = r_0, v_1 = (r_1 - v_0) m_0^-1
// mod m_1, X = v_0 + m_0 v_1 < M; the signed representative in (-M/2, M/2].
template <int K>
__device__ __forceinline__ long long garner32(const Exact32 &a, uint32_t r0, uint32_t r1)
{
    uint64_t X = r0;
    if constexpr (K == 2) {
        const uint32_t m1 = a.m[1];
        uint32_t vq = shoup32(r0, 1u, a.onep[1], m1);
        vq = vq >= m1 ? vq - m1 : vq;                               // v_0 mod m_1
        const uint32_t d = r1 >= vq ? r1 - vq : r1 + m1 - vq;
        uint32_t v1 = shoup32(d, a.inv01, a.inv01p, m1);
        v1 = v1 >= m1 ? v1 - m1 : v1;
        X += (uint64_t)v1 * a.m[0];
    }
    return X > a.half ? (long long)(X - a.M) : (long long)X;
}

template <int K>
__global__ void __launch_bounds__(256) k_exact_garner32(const __grid_constant__ Exact32 a, long long *__restrict__ h)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long n4 = a.n / 4;
    for (long long q = tid; q < n4; q += nthr) {
        const uint4 u = __ldcs(reinterpret_cast<const uint4 *>(a.rf[0]) + q);
        const uint4 w = K == 2 ? __ldcs(reinterpret_cast<const uint4 *>(a.rf[1]) + q) : make_uint4(0, 0, 0, 0);
        longlong2 *o = reinterpret_cast<longlong2 *>(h) + 2 * q;
        __stcs(o, make_longlong2(garner32<K>(a, u.x, w.x), garner32<K>(a, u.y, w.y)));
        __stcs(o + 1, make_longlong2(garner32<K>(a, u.z, w.z), garner32<K>(a, u.w, w.w)));
    }
    for (long long i = 4 * n4 + tid; i < a.n; i += nthr)
        h[i] = garner32<K>(a, a.rf[0][i], K == 2 ? a.rf[1][i] : 0u);
}

__global__ void k_exact_residues(const __grid_constant__ ExactArgs a, const long long *__restrict__ f,
                                 const long long *__restrict__ g, void *const *outf, void *const *outg)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long n4 = a.vec ? a.n / 4 : 0;
    for (int s = 0; s < 2; ++s) {
        const long long *x = s == 0 ? f : g;
        void *const *out = s == 0 ? outf : outg;
        for (long long q = tid; q < n4; q += nthr) {
            const longlong2 u0 = reinterpret_cast<const longlong2 *>(x)[2 * q];
            const longlong2 u1 = reinterpret_cast<const longlong2 *>(x)[2 * q + 1];
            const long long v[4] = {u0.x, u0.y, u1.x, u1.y};
#pragma unroll
            for (int j = 0; j < KMAX; ++j) {
                if (j >= a.k) break;
                if (a.p[j].word == 32) {
                    if (j == 0) put_residues<0, uint32_t>(a, out, 4 * q, v);
                    else if (j == 1) put_residues<1, uint32_t>(a, out, 4 * q, v);
                    else if (j == 2) put_residues<2, uint32_t>(a, out, 4 * q, v);
                    else put_residues<3, uint32_t>(a, out, 4 * q, v);
                } else {
                    if (j == 0) put_residues<0, uint64_t>(a, out, 4 * q, v);
                    else if (j == 1) put_residues<1, uint64_t>(a, out, 4 * q, v);
                    else if (j == 2) put_residues<2, uint64_t>(a, out, 4 * q, v);
                    else put_residues<3, uint64_t>(a, out, 4 * q, v);
                }
            }
        }
        for (long long i = 4 * n4 + tid; i < a.n; i += nthr) residues_scalar(a, x, out, i);
    }
}

__global__ void k_exact_garner(const __grid_constant__ ExactArgs a, const void *const *res, long long *__restrict__ h)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long n4 = a.vec ? a.n / 4 : 0;
    for (long long q = tid; q < n4; q += nthr) {
        uint64_t r[4][KMAX];
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j >= a.k) break;
            if (a.p[j].word == 32) {
                const uint4 u = reinterpret_cast<const uint4 *>(static_cast<const uint32_t *>(res[j]) + 4 * q)[0];
                r[0][j] = u.x; r[1][j] = u.y; r[2][j] = u.z; r[3][j] = u.w;
            } else {
                const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(static_cast<const uint64_t *>(res[j]) + 4 * q);
                const ulonglong2 u0 = p[0], u1 = p[1];
                r[0][j] = u0.x; r[1][j] = u0.y; r[2][j] = u1.x; r[3][j] = u1.y;
            }
        }
        longlong2 *o = reinterpret_cast<longlong2 *>(h + 4 * q);
        o[0] = make_longlong2(garner(a, r[0]), garner(a, r[1]));
        o[1] = make_longlong2(garner(a, r[2]), garner(a, r[3]));
    }
    for (long long i = 4 * n4 + tid; i < a.n; i += nthr) {
        uint64_t r[KMAX];
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j >= a.k) break;
            r[j] = load_res(a, res, j, i);
        }
        h[i] = garner(a, r);
    }
}

// Candidate primes: prime factors of Fermat numbers with ord_p(2) = 2^(n+1)
// for p | F_n (Sec. III-A, Prop. 2).  Each is re-validated by ntt_plan
// (primality, order a power of two, N | order) before use.  32-bit-word
// primes (below 2^25) come first: they run the faster path.
const uint64_t kCandidates[] = {
    13631489ull,      // F_18, Table 1
    26017793ull,      // F_12
    6700417ull,       // F_5
    2424833ull,       // F_9, Table 1
    974849ull,        // F_11
    319489ull,        // F_11, Table 1
    274177ull,        // F_6
    114689ull,        // F_12
    641ull,           // F_5, Table 1
    70525124609ull,   // F_19 (64-bit words)
    167772161ull,     // F_23
    1214251009ull,    // F_15
    825753601ull,     // F_16
    63766529ull,      // F_12
    45592577ull,      // F_10
};

}  // namespace

struct ntt_exact_s {
    uint32_t N = 0;
    uint32_t bound_bits = 0;
    int k = 0;
    ntt_plan_t plans[KMAX] = {};
    ExactArgs args{};
    double capacity_bits = 0;
    size_t wave = 0;                  // pairs per scratch wave
    void *scratch = nullptr;          // per prime: F (reused for H) and G residues of one wave
    void **ptrs_f = nullptr;          // device array of 2 KMAX pointers: F residues, then G
    void **ptrs_g = nullptr;          // ptrs_f + KMAX
    void *host_ptrs[2 * KMAX] = {};   // the same pointers, host side
    int nsm = 0;
    bool fused = false;               // whole sequences, 32-bit primes: residues and Garner fused into the convolutions
    bool all32 = false;               // every prime below 2^25: the 32-bit residue and reconstruction kernels
    Exact32 a32{};
};

extern "C" void ntt_exact_destroy(ntt_exact_t e)
{
    if (!e) return;
    for (int i = 0; i < e->k; ++i) ntt_plan_destroy(e->plans[i]);
    cudaFree(e->scratch);
    cudaFree(e->ptrs_f);             // ptrs_g points into the same allocation
    delete e;
}

extern "C" ntt_status ntt_exact_plan(uint32_t N, uint32_t bound_bits, ntt_exact_t *out)
{
    if (!out) return ntt_fail(NTT_ERR_ARG, "ntt_exact_plan: NULL out");
    *out = nullptr;
    if (N == 0 || (N & (N - 1))) return ntt_fail(NTT_ERR_LENGTH, "ntt_exact_plan: N=%u is not a power of two", N);
    if (bound_bits == 0 || bound_bits > 63)
        return ntt_fail(NTT_ERR_RANGE, "ntt_exact_plan: bound_bits=%u outside 1..63 (outputs are signed 64-bit)", bound_bits);
    ntt_exact_s *e = new ntt_exact_s();
    e->N = N;
    e->bound_bits = bound_bits;
    auto bail = [&](ntt_status s) { ntt_exact_destroy(e); return s; };
    // Greedy: candidates in order until M = prod m_i >= 2^(bound + 1), which
    // makes every h in (-2^bound, 2^bound) a distinct residue class and the
    // signed representative in (-M/2, M/2] equal to h.  M stays below 2^101.
    const u128 need = (u128)1 << (bound_bits + 1);
    u128 prod = 1;
    double bits = 0;
    for (uint64_t m : kCandidates) {
        if (e->k == KMAX || prod >= need) break;
        ntt_plan_t p = nullptr;
        if (ntt_plan(m, N, &p) != NTT_OK) continue;      // N does not divide ord_m(2), or above the supported length
        e->plans[e->k++] = p;
        prod *= m;
        bits += std::log2((double)m);
    }
    if (prod < need)
        return bail(ntt_fail(NTT_ERR_LENGTH, "ntt_exact_plan: the Rader primes available for N=%u give %.1f bits, %u + 1 needed",
                             N, bits, bound_bits));
    e->capacity_bits = bits;
    // constants
    ExactArgs &a = e->args;
    a.k = e->k;
    u128 M = 1;
    for (int i = 0; i < e->k; ++i) {
        ntt_plan_info_t info;
        ntt_plan_get_info(e->plans[i], &info);
        const uint64_t m = info.m;
        a.p[i].m = m;
        a.p[i].onep = (uint64_t)(((u128)1 << 64) / m);
        a.p[i].r64 = (uint64_t)(((u128)1 << 64) % m);
        a.p[i].word = (int)info.word_bits;
        M *= m;
    }
    for (int i = 0; i < e->k; ++i)
        for (int j = i + 1; j < e->k; ++j) {
            const uint64_t mj = a.p[j].m;
            const uint64_t c = nt::pow_mod(a.p[i].m % mj, mj - 2, mj);     // m_i^-1 mod m_j (m_j prime)
            a.inv[i][j] = c;
            a.invp[i][j] = (uint64_t)(((u128)c << 64) / mj);
        }
    const u128 half = (M - 1) / 2;
    a.half_lo = (unsigned long long)half;
    a.half_hi = (unsigned long long)(half >> 64);
    a.M_lo = (unsigned long long)M;
    a.M_hi = (unsigned long long)(M >> 64);
    // scratch: waves of pairs, at most 512 MiB of residues (8192 pairs of
    // 2^12 over two primes in one wave: fewer, fuller launches)
    size_t per_pair = 0;
    for (int i = 0; i < e->k; ++i) per_pair += 2 * (size_t)N * (a.p[i].word / 8);
    e->wave = std::min<size_t>(65536, std::max<size_t>(1, ((size_t)512 << 20) / per_pair));
    if (!ntt::dev_alloc(&e->scratch, e->wave * per_pair) ||
        !ntt::dev_alloc((void **)&e->ptrs_f, 2 * KMAX * sizeof(void *)))
        return bail(ntt_fail(NTT_ERR_OOM, "ntt_exact_plan: scratch"));
    e->ptrs_g = e->ptrs_f + KMAX;
    void *host[2 * KMAX] = {};
    unsigned char *base = (unsigned char *)e->scratch;
    for (int i = 0; i < e->k; ++i) {
        const size_t bytes = e->wave * (size_t)N * (a.p[i].word / 8);
        host[i] = base;
        host[KMAX + i] = base + bytes;
        base += 2 * bytes;
    }
    if (cudaMemcpy(e->ptrs_f, host, sizeof host, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(ntt_fail(NTT_ERR_CUDA, "ntt_exact_plan: upload"));
    memcpy(e->host_ptrs, host, sizeof host);
    e->all32 = true;
    for (int i = 0; i < e->k; ++i) e->all32 = e->all32 && a.p[i].word == 32 && a.p[i].m < (1ull << 25);
    if (e->all32) {
        Exact32 &b = e->a32;
        b.k = e->k;
        for (int i = 0; i < e->k; ++i) {
            const uint64_t m = a.p[i].m;
            b.m[i] = (uint32_t)m;
            b.c[i] = (uint32_t)((1ull << 32) % m);
            b.cp[i] = (uint32_t)(((uint64_t)b.c[i] << 32) / m);
            b.onep[i] = (uint32_t)((1ull << 32) / m);
            b.r64[i] = (uint32_t)a.p[i].r64;
            b.rf[i] = (uint32_t *)host[i];
            b.rg[i] = (uint32_t *)host[KMAX + i];
        }
        if (e->k == 2) {
            b.inv01 = (uint32_t)a.inv[0][1];
            b.inv01p = (uint32_t)(((uint64_t)b.inv01 << 32) / b.m[1]);
        }
        if (e->k <= 2) {
            b.M = (unsigned long long)M;
            b.half = (unsigned long long)half;
        }
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&e->nsm, cudaDevAttrMultiProcessorCount, dev);
    // The fused form (NTT_EXACT_FUSED=1; whole sequences, 32-bit primes only)
    // saves the residue and reconstruction passes' memory traffic, but adds
    // their arithmetic to the IMAD-bound convolution kernels: measured 1.53
    // against 0.98 ms for 8192 pairs of 2^12, so the three passes are the
    // default.
    const char *env = getenv("NTT_EXACT_FUSED");
    e->fused = env && atoi(env) != 0;
    for (int i = 0; i < e->k && e->fused; ++i) {
        ntt_plan_info_t info;
        ntt_plan_get_info(e->plans[i], &info);
        if (info.word_bits != 32 || info.four_step) e->fused = false;
    }
    *out = e;
    return NTT_OK;
}

extern "C" ntt_status ntt_exact_get_info(ntt_exact_t e, ntt_exact_info_t *info)
{
    if (!e || !info) return ntt_fail(NTT_ERR_ARG, "ntt_exact_get_info: NULL argument");
    memset(info, 0, sizeof *info);
    info->N = e->N;
    info->bound_bits = e->bound_bits;
    info->nprimes = (uint32_t)e->k;
    for (int i = 0; i < e->k; ++i) {
        info->primes[i] = e->args.p[i].m;
        info->word_bits[i] = (uint32_t)e->args.p[i].word;
    }
    info->capacity_bits = e->capacity_bits;
    info->wave = (uint64_t)e->wave;
    return NTT_OK;
}

extern "C" ntt_status conv_exact(ntt_exact_t e, const int64_t *f, const int64_t *g, int64_t *h, size_t batch,
                                 ntt_stream_t stream)
{
    if (!e || !f || !g || !h || batch == 0) return ntt_fail(NTT_ERR_ARG, "conv_exact: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 256;
    for (size_t p0 = 0; p0 < batch; p0 += e->wave) {
        const size_t np = std::min(e->wave, batch - p0);
        ExactArgs a = e->args;
        a.n = (long long)(np * e->N);
        const int grid = (int)std::min<long long>((a.n + threads - 1) / threads, (long long)e->nsm * 8);
        const size_t off = p0 * e->N;
        const long long *fw = (const long long *)f + off, *gw = (const long long *)g + off;
        long long *hw = (long long *)h + off;
        // scratch bases are 256-byte aligned and hold whole waves, so only the
        // caller's bases decide the four-element path
        if (e->fused) {
            // one fused launch per prime: int64 inputs reduced in registers;
            // the last prime reconstructs h from the others' residues
            for (int i = 0; i < e->k; ++i) {
                a.j = i;
                a.h64 = hw;
                for (int q = 0; q < KMAX; ++q) a.prev[q] = e->host_ptrs[q];
                const bool last = i == e->k - 1;
                ntt_status s = ntt_launch_exact(e->plans[i], last, fw, gw, last ? nullptr : e->host_ptrs[i], &a,
                                                (long long)np, st);
                if (s != NTT_OK) return s;
            }
            continue;
        }
        a.vec = ((((uintptr_t)fw | (uintptr_t)gw | (uintptr_t)hw) & 15u) == 0) ? 1 : 0;
        Exact32 b = e->a32;
        b.n = a.n;
        const bool fast = e->all32 && a.vec;
        if (fast) {
            switch (e->k) {
            case 1: k_exact_residues32<1><<<grid, threads, 0, st>>>(b, fw, gw); break;
            case 2: k_exact_residues32<2><<<grid, threads, 0, st>>>(b, fw, gw); break;
            case 3: k_exact_residues32<3><<<grid, threads, 0, st>>>(b, fw, gw); break;
            default: k_exact_residues32<4><<<grid, threads, 0, st>>>(b, fw, gw); break;
            }
        } else {
            k_exact_residues<<<grid, threads, 0, st>>>(a, fw, gw, e->ptrs_f, e->ptrs_g);
        }
        cudaError_t err = ntt::launched();
        if (err != cudaSuccess) return ntt_fail(NTT_ERR_CUDA, "conv_exact: residues: %s", cudaGetErrorString(err));
        for (int i = 0; i < e->k; ++i) {
            ntt_status s = conv_circular(e->plans[i], e->host_ptrs[i], e->host_ptrs[KMAX + i], e->host_ptrs[i], np, stream);
            if (s != NTT_OK) return s;
        }
        if (fast && e->k == 1) k_exact_garner32<1><<<grid, threads, 0, st>>>(b, hw);
        else if (fast && e->k == 2) k_exact_garner32<2><<<grid, threads, 0, st>>>(b, hw);
        else k_exact_garner<<<grid, threads, 0, st>>>(a, e->ptrs_f, hw);
        err = ntt::launched();
        if (err != cudaSuccess) return ntt_fail(NTT_ERR_CUDA, "conv_exact: reconstruction: %s", cudaGetErrorString(err));
    }
    return NTT_OK;
}
