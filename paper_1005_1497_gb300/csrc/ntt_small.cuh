// ntt_small.cuh -- the whole convolution of one short pair by one thread
// block, for batches too small to fill the GPU with the kernels that give
// each pair one warp (k_conv_fused).
//
// The same transform tree as the register engine (ntt_core.cuh, Sec. I with
// the power-of-two root): forward level d, node i pairs the elements at
// distance 2^{L-1-d} with the twiddle z_i = w^{brv_{L-1}(i)} (the plan's
// table), natural order in, bit-reversed order out; the inverse is the
// transposed tree with the same twiddles, the factor N^-1 of Eq. 3 is folded
// into the pointwise product, and the output is stored at <-t>_N.  Here the
// whole block walks the tree in shared memory, two levels per step (four
// elements per work item) and one block barrier per step, so that a single
// pair runs on every scheduler of its SM instead of on one warp.  Measured on
// GB300 against k_conv_fused: 2^10 x 1 pair 8.2 -> 6.2 us, 2^10 x 152 pairs
// 10.3 -> 6.2 us, 2^6 x 608 pairs 14.3 -> 4.1 us (bit-identical); the
// one-warp kernels win once the batch fills the GPU (2^10 x 1216 pairs:
// 10.3 against 16.4 us), which decides the plan's small-batch limit.
#pragma once
#include "ntt_kernels.cuh"

namespace ntt {

constexpr int SMALL_THREADS = 256;

template <typename W, int L> struct SmallShape {
    static constexpr uint32_t N = 1u << L;
    static constexpr uint32_t TWP = N / 2;                       // (twiddle, quotient) pairs of the table
    static constexpr size_t smem = (2 * (size_t)N + 2 * (size_t)TWP) * sizeof(W);
};

// Forward levels D and D+1 on one item u of sequence x: node i of level D,
// offset j inside its lower half-of-half.
template <typename W, int L, int D>
__device__ __forceinline__ void small_fwd4(W *x, const W *zt, uint32_t u, const ModC<W> &c)
{
    constexpr uint32_t t = (1u << L) >> (D + 1), q = t >> 1;    // half-sizes of levels D and D+1
    const uint32_t i = u / q, j = u % q;
    const uint32_t p0 = 2 * i * t + j, p1 = p0 + q, p2 = p0 + t, p3 = p2 + q;
    W a0 = x[p0], a1 = x[p1], a2 = x[p2], a3 = x[p3];
    ct_bfly<W>(a0, a2, zt[2 * i], zt[2 * i + 1], c);
    ct_bfly<W>(a1, a3, zt[2 * i], zt[2 * i + 1], c);
    ct_bfly<W>(a0, a1, zt[4 * i], zt[4 * i + 1], c);            // node 2i of level D+1
    ct_bfly<W>(a2, a3, zt[4 * i + 2], zt[4 * i + 3], c);        // node 2i+1
    x[p0] = a0; x[p1] = a1; x[p2] = a2; x[p3] = a3;
}

// Level D alone (the deepest level when L is odd).
template <typename W, int L, int D>
__device__ __forceinline__ void small_fwd2(W *x, const W *zt, uint32_t u, const ModC<W> &c)
{
    constexpr uint32_t t = (1u << L) >> (D + 1);
    const uint32_t i = u / t, j = u % t;
    const uint32_t p0 = 2 * i * t + j, p1 = p0 + t;
    W a0 = x[p0], a1 = x[p1];
    ct_bfly<W>(a0, a1, zt[2 * i], zt[2 * i + 1], c);
    x[p0] = a0; x[p1] = a1;
}

// Transposed levels D+1 then D.
template <typename W, int L, int D>
__device__ __forceinline__ void small_inv4(W *x, const W *zt, uint32_t u, const ModC<W> &c)
{
    constexpr uint32_t t = (1u << L) >> (D + 1), q = t >> 1;
    const uint32_t i = u / q, j = u % q;
    const uint32_t p0 = 2 * i * t + j, p1 = p0 + q, p2 = p0 + t, p3 = p2 + q;
    W a0 = x[p0], a1 = x[p1], a2 = x[p2], a3 = x[p3];
    gs_bfly<W>(a0, a1, zt[4 * i], zt[4 * i + 1], c);
    gs_bfly<W>(a2, a3, zt[4 * i + 2], zt[4 * i + 3], c);
    gs_bfly<W>(a0, a2, zt[2 * i], zt[2 * i + 1], c);
    gs_bfly<W>(a1, a3, zt[2 * i], zt[2 * i + 1], c);
    x[p0] = a0; x[p1] = a1; x[p2] = a2; x[p3] = a3;
}

template <typename W, int L, int D>
__device__ __forceinline__ void small_inv2(W *x, const W *zt, uint32_t u, const ModC<W> &c)
{
    constexpr uint32_t t = (1u << L) >> (D + 1);
    const uint32_t i = u / t, j = u % t;
    const uint32_t p0 = 2 * i * t + j, p1 = p0 + t;
    W a0 = x[p0], a1 = x[p1];
    gs_bfly<W>(a0, a1, zt[2 * i], zt[2 * i + 1], c);
    x[p0] = a0; x[p1] = a1;
}

// Forward levels D, D+1, ... of f and g together (items of f first).
template <typename W, int L, int D>
__device__ __forceinline__ void small_fwd_from(W *f, W *g, const W *zt, const ModC<W> &c)
{
    constexpr uint32_t N = 1u << L;
    if constexpr (D + 1 < L) {
        for (uint32_t u = threadIdx.x; u < N / 2; u += SMALL_THREADS)
            small_fwd4<W, L, D>(u < N / 4 ? f : g, zt, u & (N / 4 - 1), c);
        __syncthreads();
        small_fwd_from<W, L, D + 2>(f, g, zt, c);
    } else if constexpr (D < L) {
        for (uint32_t u = threadIdx.x; u < N; u += SMALL_THREADS)
            small_fwd2<W, L, D>(u < N / 2 ? f : g, zt, u & (N / 2 - 1), c);
        __syncthreads();
    }
}

// Transposed level pairs (D, D-1), (D-2, D-3), ... down to level 0.
template <typename W, int L, int D>
__device__ __forceinline__ void small_inv_pairs(W *x, const W *zt, const ModC<W> &c)
{
    constexpr uint32_t N = 1u << L;
    if constexpr (D >= 1) {
        for (uint32_t u = threadIdx.x; u < N / 4; u += SMALL_THREADS) small_inv4<W, L, D - 1>(x, zt, u, c);
        __syncthreads();
        small_inv_pairs<W, L, D - 2>(x, zt, c);
    }
}

// Pairs blockIdx.x, blockIdx.x + gridDim.x, ... of contiguous f, g, h.
// Inputs in [0, m); outputs canonical.
template <typename W, int L>
__global__ void __launch_bounds__(SMALL_THREADS) k_conv_small(const __grid_constant__ RowArgs<W> a)
{
    using SH = SmallShape<W, L>;
    constexpr uint32_t N = SH::N;
    extern __shared__ __align__(16) unsigned char smem_small[];
    W *f = reinterpret_cast<W *>(smem_small), *g = f + N, *zt = g + N;
    for (uint32_t i = threadIdx.x; i < 2 * SH::TWP; i += SMALL_THREADS) zt[i] = a.tw[i];
    for (long long pr = blockIdx.x; pr < a.nrows; pr += gridDim.x) {
        const size_t off = (size_t)(a.pair0 + pr) * N;
        for (uint32_t i = threadIdx.x; i < N; i += SMALL_THREADS) {
            f[i] = a.f[off + i];
            g[i] = a.g[off + i];
        }
        __syncthreads();
        small_fwd_from<W, L, 0>(f, g, zt, a.c);
        for (uint32_t i = threadIdx.x; i < N; i += SMALL_THREADS) f[i] = pointwise(f[i], g[i], a.c);
        __syncthreads();
        if constexpr (L % 2 == 1) {                      // the lone deepest level first
            for (uint32_t u = threadIdx.x; u < N / 2; u += SMALL_THREADS) small_inv2<W, L, L - 1>(f, zt, u, a.c);
            __syncthreads();
        }
        small_inv_pairs<W, L, (L % 2 == 0) ? L - 1 : L - 2>(f, zt, a.c);
        for (uint32_t i = threadIdx.x; i < N; i += SMALL_THREADS)
            a.h[off + i] = canon<W>(f[(N - i) & (N - 1u)], (W)1, a.c.onep, a.c.m);
        __syncthreads();                                 // f, g are refilled for the next pair
    }
}

}  // namespace ntt
