// tma_cols_probe.cu -- the split path's column passes (N = 2^19, rows of
// 2^14, 32-bit words, twist form) staged through shared memory by the TMA
// unit, against the library's plain kernels (k_cols_fwd, k_cols_inv5), which
// load each thread's column straight into registers.
//
// Staged form: one producer thread per block issues, S stages ahead, the
// copies of a tile -- RC = 32 rows x TC columns of each of the tile's
// sequences (f and g of Q pairs forward, H~ of Q pairs inverse) plus the
// tile's twist factors -- and signals their arrival on the stage's mbarrier;
// one consumer thread per (sequence, column) transforms its column out of
// shared memory, stores with plain coalesced stores, and releases the stage
// on a second mbarrier.  TILED: one cp.async.bulk.tensor.2d copy per
// sub-tile (a box of TC x 32 of the sequence viewed as [rows][2^14]);
// otherwise one untiled cp.async.bulk per row segment.  Every wait is
// bounded (about a second); a wait that runs out counts in *err and the
// block leaves after waiting, again bounded, for its copies in flight.
//
// Prints one line per kernel: "name threads blocks_per_sm ms diff err"
// (diff: output words that differ from the plain kernel's; err: waits that
// ran out).  Built and run by test_gpu_tma_cols.py:
//     tma_cols_probe <pairs> <reps>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>
#include "ntt_kernels.cuh"
#include "nt_host.h"

using namespace ntt;
constexpr int L = 19, LR = 14, LC = L - LR, RC = 1 << LC;
constexpr uint32_t N = 1u << L, C = 1u << LR;

__device__ __forceinline__ uint32_t sm_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// at most `rounds` waits of at most 20 us each
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int rounds)
{
    for (int i = 0; i < rounds; ++i) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity), "r"(20000u)
                     : "memory");
        if (ok) return true;
    }
    return false;
}
constexpr int ROUNDS = 50000;
__device__ __forceinline__ void copy_rows(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void copy_box(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}

struct Maps {
    CUtensorMap src0, src1, tbl;     // sequences viewed as [rows][2^14]; twist factors as [32][2 * 2^14]
};

template <int DIR, int Q, int TC> struct Shape {
    static constexpr int NSEQ = DIR == 0 ? 2 : 1, NSUB = NSEQ * Q, CONS = NSUB * TC, THREADS = CONS + 32;
    static constexpr uint32_t CHUNKS = C / TC, SUBB = (uint32_t)RC * TC * 4, TBLB = (uint32_t)RC * TC * 8;
    static constexpr uint32_t STAGEB = NSUB * SUBB + TBLB;
};
template <int DIR, int Q, int TC, int S> constexpr size_t smem_of() { return (size_t)S * Shape<DIR, Q, TC>::STAGEB + 16 * S + 1024; }

template <int DIR, bool TILED, int Q, int TC, int S>
__global__ void __launch_bounds__(Shape<DIR, Q, TC>::THREADS)
    k_cols_staged(const __grid_constant__ ColArgs<uint32_t> a, const __grid_constant__ Maps maps, int *err)
{
    using W = uint32_t;
    using B = Shape<DIR, Q, TC>;
    constexpr int NSEQ = B::NSEQ, CONS = B::CONS;
    extern __shared__ __align__(1024) unsigned char smem_probe[];
    unsigned char *smem = smem_probe + ((1024u - (sm_addr(smem_probe) & 1023u)) & 1023u);
    const uint32_t full0 = sm_addr(smem + (size_t)S * B::STAGEB), empty0 = full0 + 8 * S;
    const int tid = threadIdx.x;
    const long long G = (a.npairs + Q - 1) / Q, T = G * B::CHUNKS;     // tiles: chunk-major
    const long long t0 = (long long)blockIdx.x * T / gridDim.x, t1 = (long long)(blockIdx.x + 1) * T / gridDim.x;
    if (tid == 0) {
        for (int j = 0; j < S; ++j) {
            mbar_init(full0 + 8 * j, 1);
            mbar_init(empty0 + 8 * j, CONS / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid >= CONS) {                                   // producer
        if (tid != CONS) return;
        bool ok = true;
        long long i = t0;
        for (; i < t1; ++i) {
            const int it = (int)(i - t0), j = it % S;
            if (it >= S && !mbar_wait(empty0 + 8 * j, (uint32_t)(it / S - 1) & 1u, ROUNDS)) {
                ok = false;
                break;
            }
            const long long grp = i % G;
            const int c0 = (int)((i / G) * TC);
            const int nq = (int)(a.npairs - grp * Q < Q ? a.npairs - grp * Q : Q);
            const uint32_t st = sm_addr(smem + (size_t)j * B::STAGEB), bar = full0 + 8 * j;
            mbar_expect(bar, (uint32_t)(NSEQ * nq) * B::SUBB + B::TBLB);
            for (int q = 0; q < nq; ++q)
                for (int s = 0; s < NSEQ; ++s) {
                    const long long pw = grp * Q + q;
                    const uint32_t dst = st + (uint32_t)(q * NSEQ + s) * B::SUBB;
                    if constexpr (TILED) {
                        copy_box(dst, s == 0 ? &maps.src0 : &maps.src1, c0, (int)(pw * RC), bar);
                    } else {
                        const W *src = DIR == 0 ? (s == 0 ? a.src0 : a.src1) + (size_t)(a.pair0 + pw) * N
                                                : a.dst0 + (size_t)pw * N;
                        for (int k = 0; k < RC; ++k) copy_rows(dst + (uint32_t)k * TC * 4, src + c0 + (size_t)k * C, TC * 4, bar);
                    }
                }
            const uint32_t tdst = st + (uint32_t)B::NSUB * B::SUBB;
            if constexpr (TILED) {
                copy_box(tdst, &maps.tbl, 2 * c0, 0, bar);
            } else {
                for (int k = 0; k < RC; ++k) copy_rows(tdst + (uint32_t)k * TC * 8, a.pd + 2 * ((size_t)c0 + (size_t)k * C), TC * 8, bar);
            }
        }
        for (long long u = (i - S > t0 ? i - S : t0); u < i; ++u) {      // copies in flight land before leaving
            const int it = (int)(u - t0);
            ok = mbar_wait(full0 + 8 * (it % S), (uint32_t)(it / S) & 1u, ROUNDS / 8) && ok;
        }
        if (!ok) atomicAdd(err, 1);
        return;
    }
    const int sub = tid / TC, col = tid % TC, q = sub / NSEQ, s = sub % NSEQ, lane = tid & 31;
    for (long long i = t0; i < t1; ++i) {                // consumers
        const int it = (int)(i - t0), j = it % S;
        if (!mbar_wait(full0 + 8 * j, (uint32_t)(it / S) & 1u, ROUNDS)) {
            if (lane == 0) atomicAdd(err, 1);
            return;
        }
        const long long pw = (i % G) * Q + q;
        const uint32_t c0 = (uint32_t)(i / G) * TC;
        const unsigned char *st = smem + (size_t)j * B::STAGEB;
        const W *sp = reinterpret_cast<const W *>(st + (size_t)sub * B::SUBB);
        const uint2 *tp = reinterpret_cast<const uint2 *>(st + (size_t)B::NSUB * B::SUBB);
        const bool live = pw < a.npairs;                  // the same for a whole warp
        W v[RC];
        if (live) {
            if constexpr (DIR == 0) {
#pragma unroll
                for (int k = 0; k < RC; ++k) v[k] = sp[k * TC + col];
                col_fwd_levels<W, L, LR, LC - 1>(v, a.tw, a.c);
#pragma unroll
                for (int k = 0; k < RC; ++k) {
                    const uint2 z = tp[k * TC + col];
                    v[k] = csub<W>(shoup<W>(v[k], z.x, z.y, a.c.m), a.c.m);
                }
            } else {
#pragma unroll
                for (int k = 0; k < RC; ++k) {
                    const uint2 z = tp[k * TC + col];
                    v[k] = shoup<W>(sp[k * TC + col], z.x, z.y, a.c.m);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8 * j);
        if (!live) continue;
        if constexpr (DIR == 0) {
            W *dst = (s == 0 ? a.dst0 : a.dst1) + (size_t)pw * N;
#pragma unroll
            for (int k = 0; k < RC; ++k) dst[c0 + col + ((uint32_t)k << LR)] = v[k];
        } else {
            colg_levels<W, LC, 0, 0, 0, TW_GLOBAL, RC>(v, 0u, a.tw, a.c);
            W *out = a.out + (size_t)(a.pair0 + pw) * N;
#pragma unroll
            for (int k = 0; k < RC; ++k) {
                const uint32_t x = c0 + col + ((uint32_t)k << LR);
                out[(N - x) & (N - 1u)] = csub<W>(v[k], a.c.m);
            }
        }
    }
}

__global__ void k_fill(uint32_t *p, size_t n, uint32_t m, unsigned long long seed)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        unsigned long long z = seed + i * 0x9e3779b97f4a7c15ull;            // SplitMix64 finaliser
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        p[i] = (uint32_t)((z ^ (z >> 31)) % m);
    }
}
__global__ void k_diff(const uint32_t *x, const uint32_t *y, size_t n, unsigned long long *cnt)
{
    unsigned long long c = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) c += x[i] != y[i];
    if (c) atomicAdd(cnt, c);
}

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { printf("status %s (line %d)\n", cudaGetErrorString(e_), __LINE__); exit(1); } } while (0)

static CUtensorMap map2d(const void *base, uint64_t inner, uint64_t rows, uint32_t bx, uint32_t by)
{
    CUtensorMap m;
    cuuint64_t dims[2] = {inner, rows}, strides[1] = {inner * 4};
    cuuint32_t box[2] = {bx, by}, es[2] = {1, 1};
    if (cuTensorMapEncodeTiled(&m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void *>(base), dims, strides, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        printf("status tensor map encoding failed\n");
        exit(1);
    }
    return m;
}

template <typename F> static float time_ms(F f, int reps)
{
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
    for (int i = 0; i < 3; ++i) f();
    CK(cudaEventRecord(e0));
    for (int i = 0; i < reps; ++i) f();
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    return ms / reps;
}

int main(int argc, char **argv)
{
    const long long np = argc > 1 ? atoll(argv[1]) : 64;
    const int reps = argc > 2 ? atoi(argv[2]) : 20;
    const uint32_t m = 13631489;
    ModC<uint32_t> c{};
    c.m = m; c.m2 = 2 * m;
    c.mneg = (uint32_t)(0 - nt::inv_pow2(m, 32));
    c.onep = (uint32_t)nt::shoup_quot(1, m, 32);
    // node twiddles and twist factors: arbitrary residues with their Shoup
    // quotients (the kernels compared run the same arithmetic on them)
    std::mt19937_64 rng(5);
    std::vector<uint32_t> tw(N), pd(2 * (size_t)N);
    for (size_t i = 0; i < tw.size(); i += 2) { tw[i] = (uint32_t)(rng() % m); tw[i + 1] = (uint32_t)nt::shoup_quot(tw[i], m, 32); }
    for (size_t i = 0; i < pd.size(); i += 2) { pd[i] = (uint32_t)(rng() % m); pd[i + 1] = (uint32_t)nt::shoup_quot(pd[i], m, 32); }
    const size_t n = (size_t)np * N;
    uint32_t *dtw, *dpd, *f, *g, *s0, *s1, *h0, *t0, *t1, *h1;
    int *err;
    unsigned long long *cnt;
    CK(cudaMalloc(&dtw, tw.size() * 4)); CK(cudaMalloc(&dpd, pd.size() * 4));
    CK(cudaMemcpy(dtw, tw.data(), tw.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dpd, pd.data(), pd.size() * 4, cudaMemcpyHostToDevice));
    for (uint32_t **p : {&f, &g, &s0, &s1, &h0, &t0, &t1, &h1}) CK(cudaMalloc(p, n * 4));
    CK(cudaMalloc(&err, 4)); CK(cudaMemset(err, 0, 4)); CK(cudaMalloc(&cnt, 8));
    k_fill<<<1024, 256>>>(f, n, m, 1);
    k_fill<<<1024, 256>>>(g, n, m, 2);
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0));
    // the plain kernels: F~, G~ into s0, s1; h from s0 into h0
    ColArgs<uint32_t> plain{f, g, nullptr, s0, s1, h0, np, 0, dtw, c, nullptr, nullptr, dpd};
    const int grid = (int)(((np << LR) + 255) / 256);
    auto fwd = [&] { k_cols_fwd<uint32_t, L, LR, 2, 0, true><<<grid, 256>>>(plain); };
    auto inv = [&] { k_cols_inv5<uint32_t, L, LR, 0, true><<<grid, 256>>>(plain); };
    fwd(); inv();
    CK(cudaDeviceSynchronize());
    printf("plain_fwd 256 - %.4f 0 0\n", time_ms(fwd, reps));
    printf("plain_inv 256 - %.4f 0 0\n", time_ms(inv, reps));
    auto diff = [&](const uint32_t *x, const uint32_t *y) {
        CK(cudaMemset(cnt, 0, 8));
        k_diff<<<1024, 256>>>(x, y, n, cnt);
        unsigned long long d = 0;
        CK(cudaMemcpy(&d, cnt, 8, cudaMemcpyDeviceToHost));
        return d;
    };
    struct Variant {
        const char *name;
        void (*k)(ColArgs<uint32_t>, Maps, int *);
        size_t smem;
        int threads, dir, tc;
    };
    const Variant vs[] = {
        {"tiled_fwd_q1_tc128_s3", k_cols_staged<0, true, 1, 128, 3>, smem_of<0, 1, 128, 3>(), Shape<0, 1, 128>::THREADS, 0, 128},
        {"tiled_fwd_q2_tc128_s2", k_cols_staged<0, true, 2, 128, 2>, smem_of<0, 2, 128, 2>(), Shape<0, 2, 128>::THREADS, 0, 128},
        {"rows_fwd_q1_tc128_s3", k_cols_staged<0, false, 1, 128, 3>, smem_of<0, 1, 128, 3>(), Shape<0, 1, 128>::THREADS, 0, 128},
        {"tiled_inv_q2_tc128_s3", k_cols_staged<1, true, 2, 128, 3>, smem_of<1, 2, 128, 3>(), Shape<1, 2, 128>::THREADS, 1, 128},
        {"tiled_inv_q4_tc128_s2", k_cols_staged<1, true, 4, 128, 2>, smem_of<1, 4, 128, 2>(), Shape<1, 4, 128>::THREADS, 1, 128},
        {"rows_inv_q2_tc128_s3", k_cols_staged<1, false, 2, 128, 3>, smem_of<1, 2, 128, 3>(), Shape<1, 2, 128>::THREADS, 1, 128},
    };
    for (const Variant &v : vs) {
        CK(cudaFuncSetAttribute(v.k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem));
        int per = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, v.k, v.threads, v.smem));
        if (per < 1) { printf("status no residency for %s\n", v.name); return 1; }
        Maps mp;
        if (v.dir == 0) {
            mp.src0 = map2d(f, C, (uint64_t)np * RC, v.tc, RC);
            mp.src1 = map2d(g, C, (uint64_t)np * RC, v.tc, RC);
        } else {
            mp.src0 = map2d(s0, C, (uint64_t)np * RC, v.tc, RC);
            mp.src1 = mp.src0;
        }
        mp.tbl = map2d(dpd, 2 * (uint64_t)C, RC, 2 * v.tc, RC);
        ColArgs<uint32_t> arg{f, g, nullptr, v.dir == 0 ? t0 : s0, t1, h1, np, 0, dtw, c, nullptr, nullptr, dpd};
        CK(cudaMemset(t0, 0, n * 4)); CK(cudaMemset(t1, 0, n * 4)); CK(cudaMemset(h1, 0, n * 4)); CK(cudaMemset(err, 0, 4));
        const int g2 = nsm * per;
        v.k<<<g2, v.threads, v.smem>>>(arg, mp, err);
        CK(cudaDeviceSynchronize());
        const unsigned long long d = v.dir == 0 ? diff(s0, t0) + diff(s1, t1) : diff(h0, h1);
        const float ms = time_ms([&] { v.k<<<g2, v.threads, v.smem>>>(arg, mp, err); }, reps);
        int e = 0;
        CK(cudaMemcpy(&e, err, 4, cudaMemcpyDeviceToHost));
        printf("%s %d %d %.4f %llu %d\n", v.name, v.threads, per, ms, d, e);
    }
    CK(cudaGetLastError());
    printf("status %s\n", cudaGetErrorString(cudaDeviceSynchronize()));
    return 0;
}
