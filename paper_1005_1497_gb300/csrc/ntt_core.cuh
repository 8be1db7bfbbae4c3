// ntt_core.cuh -- device arithmetic and the register/shared-memory transform
// engine of the exact digital convolution (Chandra, "Fast Digital
// Convolutions using Bit-Shifts", Eq. 1-3).
//
// Transform structure.  The forward transform is the radix-2 Cooley-Tukey
// algorithm of Sec. I with e^{2 pi i a/N} replaced by powers of the integer
// root w = 2^(N_Max/N): it is evaluated as the tree of "node" splits
//     level d, node i:  (a, b) -> (a + z_i b, a - z_i b),  z_i = w^{brv_{L-1}(i)}
// over butterfly pairs at distance 2^{L-1-d}, natural order in, bit-reversed
// order out.  Every level's twiddles are the first 2^d entries of ONE table
// z_i (i < N/2), so a single table of powers of two serves all levels.
//
// The inverse transform is the transpose of that tree (same twiddles,
// butterflies (a, b) -> (a + b, z_i (a - b)), levels in reverse order),
// which maps the bit-reversed spectrum back to natural order and computes
// the forward transform F applied to the spectrum.  Because
// F^{-1} = N^{-1} R F with (R v)(t) = v(<-t>_N) (Eq. 3 with w^{-ut} =
// w^{<-ut>_N}), the output is stored at index <-t>_N and the factor N^-1 is
// folded into the pointwise product.
//
// Arithmetic.  Residues are kept "lazy": a twiddle product uses Shoup's
// precomputed quotient z' = floor(z 2^B / m) and returns a value in [0, 2m)
// for ANY input below 2^B, so the forward butterflies never reduce their
// sums: after d levels every value is below 2 m (d + 1).  The inverse
// butterflies reduce their sums with one conditional subtraction.  The
// pointwise product is a Shoup product by N^-1 2^B followed by a Montgomery
// reduction (R = 2^B), which yields F G N^-1 mod m in [0, 2m).  Final outputs
// are reduced to the canonical range [0, m).  B is the word width (32/64).
//
// Thread mapping.  A "row" of 2^LR elements is transformed by a group of T
// threads, each holding R = 2^RL elements in registers.  The levels are
// processed in passes of up to RL bits, from the top bit down.  In pass p the
// register index k (RL bits) selects element bits [lo_p, lo_p + RL) and the
// thread index supplies the remaining bits, low bits first, so consecutive
// lanes touch consecutive elements whenever lo_p >= 5.  Between passes the
// group exchanges its row through shared memory, padded by one word every
// 2^PADSH words, which makes every pass's accesses free of bank conflicts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ntt {

template <typename W> struct Arith;

template <> struct Arith<uint32_t> {
    static constexpr int RB = 5;        // log2 of elements held per thread
    static constexpr int BITS = 32;
    static constexpr int PADSH = 5;     // one pad word per 32 words
    __device__ __forceinline__ static uint32_t mulhi(uint32_t a, uint32_t b) { return __umulhi(a, b); }
};

template <> struct Arith<uint64_t> {
    static constexpr int RB = 4;
    static constexpr int BITS = 64;
    static constexpr int PADSH = 4;     // one pad word per 16 eight-byte words
    __device__ __forceinline__ static uint64_t mulhi(uint64_t a, uint64_t b) { return __umul64hi(a, b); }
};

// Per-plan constants, passed by value in the kernel parameters.
template <typename W> struct ModC {
    W m;        // modulus
    W m2;       // 2 m
    W mneg;     // -m^{-1} mod 2^B (Montgomery)
    W cN;       // N^{-1} 2^B mod m (pointwise factor)
    W cNp;      // floor(cN 2^B / m)
    W onep;     // floor(2^B / m): Shoup quotient of the factor 1
    W ninv;     // N^{-1} mod m
    W ninvp;    // floor(ninv 2^B / m)
};

// Shoup product: b z mod m in [0, 2m) for any b < 2^B, given zp = floor(z 2^B / m).
template <typename W>
__device__ __forceinline__ W shoup(W b, W z, W zp, W m)
{
    W q = Arith<W>::mulhi(b, zp);
    return b * z - q * m;
}

// v in [0, 2m) -> [0, m)
template <typename W>
__device__ __forceinline__ W csub(W v, W m) { W t = v - m; return t < v ? t : v; }

// Forward (Cooley-Tukey) node butterfly, lazy: outputs < bound(a) + 2m.
template <typename W>
__device__ __forceinline__ void ct_bfly(W &a, W &b, W z, W zp, const ModC<W> &c)
{
    W t = shoup<W>(b, z, zp, c.m);
    W a0 = a;
    a = a0 + t;
    b = a0 - t + c.m2;
}

// Level 0 of the forward tree has only the factor 1; inputs are < m.
template <typename W>
__device__ __forceinline__ void ct_bfly_one(W &a, W &b, const ModC<W> &c)
{
    W a0 = a;
    a = a0 + b;
    b = a0 - b + c.m;
}

// Butterfly with the twiddle 1 on inputs bounded by B (B a multiple of m):
// outputs < 2B, no product.  Used where the twiddle is known to be 1 at
// compile time (node 0 of a forward level, position 0 of an inverse level)
// and the doubled bound still fits the word (see the bound notes below).
template <typename W>
__device__ __forceinline__ void ct_bfly_unit(W &a, W &b, W B)
{
    W a0 = a;
    a = a0 + b;
    b = a0 - b + B;
}

// Transposed (Gentleman-Sande) node butterfly on inputs < 2m; outputs < 2m.
template <typename W>
__device__ __forceinline__ void gs_bfly(W &a, W &b, W z, W zp, const ModC<W> &c)
{
    W s = a + b;
    W d = a - b + c.m2;
    W s2 = s - c.m2;
    a = s2 < s ? s2 : s;
    b = shoup<W>(d, z, zp, c.m);
}

template <typename W>
__device__ __forceinline__ void gs_bfly_one(W &a, W &b, const ModC<W> &c)
{
    W s = a + b;
    W d = a - b + c.m2;
    W s2 = s - c.m2, d2 = d - c.m2;
    a = s2 < s ? s2 : s;
    b = d2 < d ? d2 : d;
}

// Pointwise product F G N^{-1} mod m in [0, 2m): Shoup by N^{-1} 2^B, then a
// Montgomery reduction of the double-word product.
__device__ __forceinline__ uint32_t pointwise(uint32_t F, uint32_t G, const ModC<uint32_t> &c)
{
    uint32_t u = shoup<uint32_t>(F, c.cN, c.cNp, c.m);
    uint32_t lo = u * G;
    uint32_t hi = __umulhi(u, G);
    uint32_t q = lo * c.mneg;
    return hi + __umulhi(q, c.m) + (lo != 0u ? 1u : 0u);
}

__device__ __forceinline__ uint64_t pointwise(uint64_t F, uint64_t G, const ModC<uint64_t> &c)
{
    uint64_t u = shoup<uint64_t>(F, c.cN, c.cNp, c.m);
    uint64_t lo = u * G;
    uint64_t hi = __umul64hi(u, G);
    uint64_t q = lo * c.mneg;
    return hi + __umul64hi(q, c.m) + (lo != 0ull ? 1ull : 0ull);
}

// ---------------------------------------------------------------- geometry

template <typename W, int LR_>
struct Geo {
    static constexpr int LR = LR_;
    static constexpr int RB = Arith<W>::RB;
    static constexpr int RL = LR < RB ? LR : RB;
    static constexpr int R = 1 << RL;                   // elements per thread
    static constexpr int TL = LR - RL;
    static constexpr int T = 1 << TL;                   // threads per row
    static constexpr int NPASS = LR <= RB ? 1 : (LR + RB - 1) / RB;
    static constexpr int PADSH = Arith<W>::PADSH;
    static constexpr int ROW = 1 << LR;
    static constexpr int ROWP = ROW + (ROW >> PADSH);   // padded words of one row region
    __host__ __device__ static constexpr int hi(int p) { return LR - p * RB; }
    __host__ __device__ static constexpr int nb(int p) { return hi(p) >= RB ? RB : hi(p); }
    __host__ __device__ static constexpr int lo(int p) { return hi(p) - nb(p); }
    // element index of (thread tau, register k) in pass p, without the row offset
    __host__ __device__ static constexpr uint32_t base(int p, uint32_t tau)
    {
        return (tau & ((1u << lo(p)) - 1u)) | ((tau >> lo(p)) << (lo(p) + RL));
    }
    __host__ __device__ static constexpr uint32_t pad(uint32_t x) { return x + (x >> PADSH); }
};

// Group synchronisation: a named barrier per multi-warp group, warp sync
// otherwise.  T threads per group; gid = group index in the block.
template <int T>
__device__ __forceinline__ void group_sync(int gid)
{
    if constexpr (T >= 64) {
        asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(T) : "memory");
    } else if constexpr (T == 32) {
        __syncwarp();
    } else if constexpr (T > 1) {
        unsigned lane = threadIdx.x & 31u;
        unsigned mask = ((1u << T) - 1u) << (lane & ~(unsigned)(T - 1));
        __syncwarp(mask);
    }
}

// Twiddle sources.  TW_GLOBAL: the plan's table in device memory, read
// through the read-only cache.  TW_SMEM: a copy in shared memory laid out in
// 16-byte chunks with an XOR swizzle: chunk c of 128-byte row r is stored at
// position c ^ fold(r), fold(r) = XOR of the 3-bit groups of r.  Folding all
// row bits (not just the low three) keeps every level's per-thread runs on
// distinct banks, including the inverse's runs whose rows are bit-reversed
// thread indices and so differ only in high bits.
enum { TW_GLOBAL = 0, TW_SMEM = 1 };

__host__ __device__ constexpr uint32_t tw_fold(uint32_t row)
{
    return (row ^ (row >> 3) ^ (row >> 6) ^ (row >> 9) ^ (row >> 12) ^ (row >> 15)) & 7u;
}
__host__ __device__ constexpr uint32_t tw_swz(uint32_t chunk) { return chunk ^ tw_fold(chunk >> 3); }

// Pairs per 16-byte chunk of the table.
template <typename W> __host__ __device__ constexpr int tw_per_chunk() { return (int)(16 / (2 * sizeof(W))); }

// Load CH (1 or 2 for 32-bit words, 1 for 64-bit words) consecutive pairs
// starting at index i (aligned to CH).
// Entry nb + t0 of the table (t0 a constant after unrolling).  The global
// path forms the 64-bit address of entry nb once and adds t0 as a pointer
// offset, so that the unrolled loads of one level share one base register
// and differ by immediates (a 32-bit nb + t0 widened afterwards cannot be
// split that way, and costs a 64-bit address per load).
template <typename W, int CH, int TWS>
__device__ __forceinline__ void load_tw(const W *__restrict__ tw, uint32_t nb, uint32_t t0, W (&z)[CH], W (&zp)[CH])
{
    constexpr int PC = tw_per_chunk<W>();
    static_assert(CH <= PC, "one chunk at most");
    const uint32_t i = nb + t0;
    if constexpr (TWS == TW_SMEM) {
        const uint32_t c = tw_swz(i / PC);
        if constexpr (sizeof(W) == 4 && CH == 2) {
            uint4 q = reinterpret_cast<const uint4 *>(tw)[c];
            z[0] = (W)q.x; zp[0] = (W)q.y; z[1] = (W)q.z; zp[1] = (W)q.w;
        } else if constexpr (sizeof(W) == 4) {
            uint2 q = reinterpret_cast<const uint2 *>(tw)[2 * c + (i & 1u)];
            z[0] = (W)q.x; zp[0] = (W)q.y;
        } else {
            ulonglong2 q = reinterpret_cast<const ulonglong2 *>(tw)[c];
            z[0] = (W)q.x; zp[0] = (W)q.y;
        }
    } else {
        const W *p = tw + 2 * (size_t)nb;                   // entry nb; + 2 t0 below
        if constexpr (sizeof(W) == 4 && CH == 2) {
            uint4 q = __ldg(reinterpret_cast<const uint4 *>(p + 2 * (size_t)t0));   // nb + t0 even
            z[0] = (W)q.x; zp[0] = (W)q.y; z[1] = (W)q.z; zp[1] = (W)q.w;
        } else if constexpr (sizeof(W) == 4) {
            uint2 q = __ldg(reinterpret_cast<const uint2 *>(p + 2 * (size_t)t0));
            z[0] = (W)q.x; zp[0] = (W)q.y;
        } else {
            ulonglong2 q = __ldg(reinterpret_cast<const ulonglong2 *>(p + 2 * (size_t)t0));
            z[0] = (W)q.x; zp[0] = (W)q.y;
        }
    }
}

// Copy the first `pairs` entries of the plan's table into shared memory in
// the swizzled layout (whole block cooperates; caller syncs afterwards).
template <typename W>
__device__ __forceinline__ void stage_twiddles(const W *__restrict__ tw, W *stw, uint32_t pairs)
{
    constexpr int PC = tw_per_chunk<W>();
    const uint32_t chunks = (pairs + PC - 1) / PC;
    for (uint32_t c = threadIdx.x; c < chunks; c += blockDim.x) {
        if (PC == 2 && pairs == 1) {
            reinterpret_cast<uint2 *>(stw)[0] = __ldg(reinterpret_cast<const uint2 *>(tw));
        } else {
            reinterpret_cast<uint4 *>(stw)[tw_swz(c)] = __ldg(reinterpret_cast<const uint4 *>(tw) + c);
        }
    }
}

// One forward level: element bit b = lo_P + JJ, global level L-1-b.
// Z0: the node base of this pass is known to be 0 (first pass of a whole
// sequence), so node 0 has the twiddle 1.  Bound note: inputs < m, level 0
// leaves < 2m and every node-0 butterfly of levels 1..4 doubles the bound
// (< 2^(d+1) m after level d), the others add 2m: at most 32m + 2m (L - 5)
// after the forward, below 50m for L <= 14.
template <typename W, int L, int LR, int P, int JJ, int NS, int TWS, bool Z0 = false>
__device__ __forceinline__ void fwd_level(W (&v)[NS][Geo<W, LR>::R], uint32_t xbase,
                                          const W *__restrict__ tw, const ModC<W> &c)
{
    using G = Geo<W, LR>;
    constexpr int R = G::R;
    constexpr int b = G::lo(P) + JJ;
    constexpr int dg = L - 1 - b;
    if constexpr (dg == 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (k & (1 << JJ)) continue;
#pragma unroll
            for (int s = 0; s < NS; ++s) ct_bfly_one<W>(v[s][k], v[s][k | (1 << JJ)], c);
        }
    } else {
        constexpr int CNT = R >> (JJ + 1);      // distinct nodes touched by this thread
        constexpr int CH = (CNT >= 2 && tw_per_chunk<W>() == 2) ? 2 : 1;
        constexpr bool UNIT0 = Z0 && P == 0 && dg <= 4;
        const uint32_t nb = xbase >> (b + 1);   // aligned to CNT
#pragma unroll
        for (int t0 = 0; t0 < CNT; t0 += CH) {
            W z[CH], zp[CH];
            load_tw<W, CH, TWS>(tw, nb, (uint32_t)t0, z, zp);
#pragma unroll
            for (int tt = 0; tt < CH; ++tt)
#pragma unroll
                for (int j = 0; j < (1 << JJ); ++j) {
                    const int k = ((t0 + tt) << (JJ + 1)) | j;
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        if (UNIT0 && t0 + tt == 0) ct_bfly_unit<W>(v[s][k], v[s][k | (1 << JJ)], c.m << dg);
                        else ct_bfly<W>(v[s][k], v[s][k | (1 << JJ)], z[tt], zp[tt], c);
                    }
                }
        }
    }
}

// Forward levels of pass P, highest element bit first.
template <typename W, int L, int LR, int P, int JJ, int NS, int TWS, bool Z0>
__device__ __forceinline__ void fwd_levels(W (&v)[NS][Geo<W, LR>::R], uint32_t xbase,
                                           const W *__restrict__ tw, const ModC<W> &c)
{
    if constexpr (JJ >= 0) {
        fwd_level<W, L, LR, P, JJ, NS, TWS, Z0>(v, xbase, tw, c);
        fwd_levels<W, L, LR, P, JJ - 1, NS, TWS, Z0>(v, xbase, tw, c);
    }
}

template <typename W, int L, int LR, int P, int NS, int TWS, bool Z0 = false>
__device__ __forceinline__ void fwd_pass(W (&v)[NS][Geo<W, LR>::R], uint32_t xbase,
                                         const W *__restrict__ tw, const ModC<W> &c)
{
    fwd_levels<W, L, LR, P, Geo<W, LR>::nb(P) - 1, NS, TWS, Z0>(v, xbase, tw, c);
}

// One transposed (inverse-direction) level.
template <typename W, int L, int LR, int P, int JJ, int TWS>
__device__ __forceinline__ void inv_level(W (&v)[Geo<W, LR>::R], uint32_t xbase,
                                          const W *__restrict__ tw, const ModC<W> &c)
{
    using G = Geo<W, LR>;
    constexpr int R = G::R;
    constexpr int b = G::lo(P) + JJ;
    constexpr int dg = L - 1 - b;
    if constexpr (dg == 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (k & (1 << JJ)) continue;
            gs_bfly_one<W>(v[k], v[k | (1 << JJ)], c);
        }
    } else {
        constexpr int CNT = R >> (JJ + 1);
        constexpr int CH = (CNT >= 2 && tw_per_chunk<W>() == 2) ? 2 : 1;
        const uint32_t nb = xbase >> (b + 1);
#pragma unroll
        for (int t0 = 0; t0 < CNT; t0 += CH) {
            W z[CH], zp[CH];
            load_tw<W, CH, TWS>(tw, nb, (uint32_t)t0, z, zp);
#pragma unroll
            for (int tt = 0; tt < CH; ++tt)
#pragma unroll
                for (int j = 0; j < (1 << JJ); ++j) {
                    const int k = ((t0 + tt) << (JJ + 1)) | j;
                    gs_bfly<W>(v[k], v[k | (1 << JJ)], z[tt], zp[tt], c);
                }
        }
    }
}

// Transposed levels of pass P, lowest element bit (deepest level) first.
template <typename W, int L, int LR, int P, int JJ, int TWS>
__device__ __forceinline__ void inv_levels(W (&v)[Geo<W, LR>::R], uint32_t xbase,
                                           const W *__restrict__ tw, const ModC<W> &c)
{
    if constexpr (JJ < Geo<W, LR>::nb(P)) {
        inv_level<W, L, LR, P, JJ, TWS>(v, xbase, tw, c);
        inv_levels<W, L, LR, P, JJ + 1, TWS>(v, xbase, tw, c);
    }
}

template <typename W, int L, int LR, int P, int TWS>
__device__ __forceinline__ void inv_pass(W (&v)[Geo<W, LR>::R], uint32_t xbase,
                                         const W *__restrict__ tw, const ModC<W> &c)
{
    inv_levels<W, L, LR, P, 0, TWS>(v, xbase, tw, c);
}

// ---- inverse direction, decimation in time -------------------------------
//
// The textbook iterative radix-2 algorithm of Sec. I, (a, b) -> (a + z b,
// a - z b) over half-lengths 2^l = 1, 2, 4, ..., takes the bit-reversed
// spectrum left by the forward tree to natural order and computes F applied
// to it; F^{-1} = N^{-1} R F (Eq. 3) then needs the output index <-t>_N and
// the factor N^-1.  Its twiddle for the pair (x, x + 2^l) is w^{(x mod 2^l)
// N / 2^(l+1)} = z_{brv_l(x mod 2^l)}: the same table, read as one
// contiguous run per thread and level.  Sums grow additively like the
// forward ones, so no butterfly reduces: inputs < 2m leave the level l = 0
// below 4m and every further level adds 2m.

template <int J>
__host__ __device__ constexpr int brv_c(int j)
{
    int r = 0;
    for (int i = 0; i < J; ++i) r |= ((j >> i) & 1) << (J - 1 - i);
    return r;
}

// Level l = lo_P + JJ of the inverse on one sequence.  In the first pass
// (lo = 0) every thread's run starts at entry 0, whose twiddle is 1: those
// butterflies skip the product.  Bound note: inputs < 2m, level 0 leaves
// < 4m, the unit butterflies of levels 1..4 double it (< 2^(l+2) m after
// level l), the others add 2m: at most 64m + 2m (L - 5), below 82m for
// L <= 14, and the final Shoup reduction accepts any word.
template <typename W, int LR, int P, int JJ, int TWS>
__device__ __forceinline__ void dit_level(W (&v)[Geo<W, LR>::R], uint32_t xbase,
                                          const W *__restrict__ tw, const ModC<W> &c)
{
    using G = Geo<W, LR>;
    constexpr int R = G::R, lo = G::lo(P);
    constexpr int l = lo + JJ;
    if constexpr (l == 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (k & 1) continue;
            W a0 = v[k];
            v[k] = a0 + v[k + 1];
            v[k + 1] = a0 - v[k + 1] + c.m2;
        }
    } else {
        constexpr int CNT = 1 << JJ;                  // distinct twiddles of this level
        constexpr int CH = (CNT >= 2 && tw_per_chunk<W>() == 2) ? 2 : 1;
        uint32_t tlo = 0;
        if constexpr (lo > 0) tlo = __brev(xbase & ((1u << lo) - 1u)) >> (32 - lo);
        const uint32_t run = tlo << JJ;               // aligned to CNT
#pragma unroll
        for (int t0 = 0; t0 < CNT; t0 += CH) {
            W z[CH], zp[CH];
            load_tw<W, CH, TWS>(tw, run, (uint32_t)t0, z, zp);
#pragma unroll
            for (int tt = 0; tt < CH; ++tt) {
                const int j = brv_c<JJ>(t0 + tt);         // register bits below JJ
#pragma unroll
                for (int hi = 0; hi < (R >> (JJ + 1)); ++hi) {
                    const int k = (hi << (JJ + 1)) | j;
                    if (lo == 0 && l <= 4 && t0 + tt == 0) ct_bfly_unit<W>(v[k], v[k | (1 << JJ)], c.m << (l + 1));
                    else ct_bfly<W>(v[k], v[k | (1 << JJ)], z[tt], zp[tt], c);
                }
            }
        }
    }
}

template <typename W, int LR, int P, int JJ, int TWS>
__device__ __forceinline__ void dit_levels(W (&v)[Geo<W, LR>::R], uint32_t xbase,
                                           const W *__restrict__ tw, const ModC<W> &c)
{
    if constexpr (JJ < Geo<W, LR>::nb(P)) {
        dit_level<W, LR, P, JJ, TWS>(v, xbase, tw, c);
        dit_levels<W, LR, P, JJ + 1, TWS>(v, xbase, tw, c);
    }
}

// Store the registers of NS sequences in the layout of pass P into the
// group's shared regions (stride ROWP words), sync, read back in pass Q.
template <typename W, int LR, int P, int Q, int NS>
__device__ __forceinline__ void exchange(W (&v)[NS][Geo<W, LR>::R], W *S, uint32_t tau, int gid)
{
    using G = Geo<W, LR>;
    constexpr int R = G::R;
    const uint32_t bp = G::pad(G::base(P, tau));
    const uint32_t bq = G::pad(G::base(Q, tau));
    group_sync<G::T>(gid);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int k = 0; k < R; ++k)
            S[s * G::ROWP + bp + G::pad((uint32_t)k << G::lo(P))] = v[s][k];
    group_sync<G::T>(gid);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int k = 0; k < R; ++k)
            v[s][k] = S[s * G::ROWP + bq + G::pad((uint32_t)k << G::lo(Q))];
}

// All forward passes P = FROM .. NPASS-1 (registers start in layout FROM).
template <typename W, int L, int LR, int P, int NS, int TWS, bool Z0 = false>
__device__ __forceinline__ void fwd_all(W (&v)[NS][Geo<W, LR>::R], uint32_t rowoff, uint32_t tau,
                                        W *S, int gid, const W *__restrict__ tw, const ModC<W> &c)
{
    using G = Geo<W, LR>;
    fwd_pass<W, L, LR, P, NS, TWS, Z0>(v, rowoff + G::base(P, tau), tw, c);
    if constexpr (P + 1 < G::NPASS) {
        exchange<W, LR, P, P + 1, NS>(v, S, tau, gid);
        fwd_all<W, L, LR, P + 1, NS, TWS, Z0>(v, rowoff, tau, S, gid, tw, c);
    }
}

// Single-sequence exchange (inverse direction).
template <typename W, int LR, int P, int Q>
__device__ __forceinline__ void exchange1(W (&v)[Geo<W, LR>::R], W *S, uint32_t tau, int gid)
{
    using G = Geo<W, LR>;
    constexpr int R = G::R;
    const uint32_t bp = G::pad(G::base(P, tau));
    const uint32_t bq = G::pad(G::base(Q, tau));
    group_sync<G::T>(gid);
#pragma unroll
    for (int k = 0; k < R; ++k) S[bp + G::pad((uint32_t)k << G::lo(P))] = v[k];
    group_sync<G::T>(gid);
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = S[bq + G::pad((uint32_t)k << G::lo(Q))];
}

// All inverse passes P = FROM .. 0 (registers start in layout FROM).
template <typename W, int L, int LR, int P, int TWS>
__device__ __forceinline__ void inv_all(W (&v)[Geo<W, LR>::R], uint32_t rowoff, uint32_t tau,
                                        W *S, int gid, const W *__restrict__ tw, const ModC<W> &c)
{
    using G = Geo<W, LR>;
    inv_pass<W, L, LR, P, TWS>(v, rowoff + G::base(P, tau), tw, c);
    if constexpr (P > 0) {
        exchange1<W, LR, P, P - 1>(v, S, tau, gid);
        inv_all<W, L, LR, P - 1, TWS>(v, rowoff, tau, S, gid, tw, c);
    }
}

// All inverse passes, decimation in time, P = FROM .. 0.
template <typename W, int LR, int P, int TWS>
__device__ __forceinline__ void dit_all(W (&v)[Geo<W, LR>::R], uint32_t rowoff, uint32_t tau,
                                        W *S, int gid, const W *__restrict__ tw, const ModC<W> &c)
{
    using G = Geo<W, LR>;
    dit_levels<W, LR, P, 0, TWS>(v, rowoff + G::base(P, tau), tw, c);
    if constexpr (P > 0) {
        exchange1<W, LR, P, P - 1>(v, S, tau, gid);
        dit_all<W, LR, P - 1, TWS>(v, rowoff, tau, S, gid, tw, c);
    }
}

// Final canonical residue of a lazily bounded value: Shoup product by the
// factor (z, zp) (1 or N^-1) into [0, 2m), then one conditional subtraction.
template <typename W>
__device__ __forceinline__ W canon(W v, W z, W zp, W m) { return csub<W>(shoup<W>(v, z, zp, m), m); }

}  // namespace ntt
