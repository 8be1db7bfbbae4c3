// ntt_kernels.cuh -- kernels of the exact digital convolution, templated on
// the word type W (uint32_t / uint64_t) and on log2 N.
#pragma once

#include "ntt_core.cuh"
#include "ntt_exact.cuh"

namespace ntt {

constexpr int BLOCK = 512;                 // threads of every row-kernel block (default)
// The whole-sequence fused kernels also come with BLK = 256: half the rows
// in flight and half the shared memory per block, so two blocks share an SM
// and pass through their barrier-separated phases independently; the
// autotuner picks per length (BLOCK for the longest whole length, whose
// rows need 512 threads).
constexpr int BLOCK_HALF = 256;

template <typename W> struct LRMax;        // longest row one block transforms
template <> struct LRMax<uint32_t> { static constexpr int v = 14; };
template <> struct LRMax<uint64_t> { static constexpr int v = 13; };

// One convolution of an uneven batch, as seen by the device.
template <typename W> struct DevDesc {
    const W *f;
    const W *g;
    W *h;
};

// Arguments of the row kernels.  For a whole-sequence launch (L == LR) row
// rho is pair pair0 + rho of the batch (contiguous arrays f, g, h or the
// descriptor list).  For the split path (L > LR) rho counts rows of the
// current wave inside the scratch arrays f (= F~, overwritten by H~) and g.
template <typename W> struct RowArgs {
    const W *f;
    const W *g;
    W *h;
    const DevDesc<W> *descs;
    long long nrows;
    long long pair0;
    const W *tw;
    ModC<W> c;
};

// Shared-memory copy of the twiddle table of a whole-sequence kernel (N/2 pairs).
template <typename W, int L>
struct TwBytes {
    static constexpr uint32_t pairs = L >= 1 ? (1u << (L - 1)) : 1u;
    static constexpr size_t v = ((size_t)pairs * 2 * sizeof(W) + 15) / 16 * 16;
};

template <typename W, int L, int LR, int BLK = BLOCK>
struct RowShape {
    using G = Geo<W, LR>;
    static constexpr int GPC = BLK / G::T;     // rows in flight per block
    static constexpr size_t smem(int ns) { return (size_t)GPC * ns * G::ROWP * sizeof(W); }
};

// Hint: fetch `bytes` bytes at p into L2 with one bulk copy-engine
// request (no registers, no shared memory).  Skipped unless 16-byte aligned.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    if (((uintptr_t)p & 15u) == 0 && bytes >= 16)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes & ~15u) : "memory");
}

// Input and output of the fused bodies: plain words (the default), or the
// ends of the exact convolution fused in -- signed 64-bit inputs reduced
// modulo the launch's prime (IN64), and for the last prime the Chinese
// remainder reconstruction of each output from the earlier primes'
// residues (GARNER), written as a signed 64-bit integer.
struct NoExact { static constexpr bool IN64 = false, GARNER = false; };
struct ExactResidues { static constexpr bool IN64 = true, GARNER = false; };
struct ExactGarner { static constexpr bool IN64 = true, GARNER = true; };

// Element i of a sequence whose first element is at base.
template <class X, typename W>
__device__ __forceinline__ W ld_elem(const W *base, uint32_t i, const ExactArgs *xa)
{
    if constexpr (X::IN64) return (W)residue(reinterpret_cast<const long long *>(base)[i], xa->p[xa->j]);
    else return base[i];
}

// Sequence `pair` of a contiguous batch of words (or of signed 64-bit words).
template <class X, typename W>
__device__ __forceinline__ const W *seq_base(const W *batch, long long pair, uint32_t N)
{
    if constexpr (X::IN64) return reinterpret_cast<const W *>(reinterpret_cast<const long long *>(batch) + (size_t)pair * N);
    else return batch + (size_t)pair * N;
}

// Canonical output r at index idx of sequence `pair` (hp: that sequence's words).
template <class X, typename W>
__device__ __forceinline__ void st_out(W *hp, long long pair, uint32_t N, uint32_t idx, W r, const ExactArgs *xa)
{
    if constexpr (X::GARNER) {
        const size_t at = (size_t)pair * N + idx;
        uint64_t rr[XKMAX];
#pragma unroll
        for (int q = 0; q < XKMAX; ++q) {
            if (q >= xa->k) break;
            rr[q] = q == xa->j ? (uint64_t)r : load_res(*xa, xa->prev, q, (long long)at);
        }
        xa->h64[at] = garner(*xa, rr);
    } else {
        hp[idx] = r;
    }
}

// Fused convolution of whole sequences (L <= LR_max), persistent.  The block
// stages the twiddle table in shared memory once.  Per pair, f and g are
// transformed together (one set of twiddle reads serves both) through shared
// regions 0 and 1, multiplied pointwise, and sent back through region 0 by
// the decimation-in-time inverse; results are stored canonical at <-x>_N.
// At the start of each pair one thread asks the copy engine to bring the
// next pair's f and g into L2, so their loads do not wait on HBM.
// Rows [base + group, a.nrows) by steps of stride.
template <typename W, int L, int SRC, class X = NoExact>
__device__ __forceinline__ void conv_fused_body(const RowArgs<W> &a, long long base, long long stride,
                                                const ExactArgs *xa = nullptr)
{
    using G = Geo<W, L>;
    constexpr int T = G::T, R = G::R, GPC = RowShape<W, L, L>::GPC;
    constexpr uint32_t N = 1u << L;
    constexpr int last = G::NPASS - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gid = threadIdx.x / T;
    const uint32_t tau = threadIdx.x % T;
    W *stw = reinterpret_cast<W *>(smem_raw);
    W *S = reinterpret_cast<W *>(smem_raw + TwBytes<W, L>::v) + (size_t)gid * 2 * G::ROWP;
    const uint32_t b0 = G::base(0, tau);
    constexpr int lo0 = G::lo(0);
    stage_twiddles<W>(a.tw, stw, TwBytes<W, L>::pairs);
    __syncthreads();

    auto ptrs = [&](long long rho, const W *&fp, const W *&gp, W *&hp) {
        const long long pair = a.pair0 + rho;
        if constexpr (SRC == 1) {
            const DevDesc<W> d = a.descs[pair];
            fp = d.f; gp = d.g; hp = d.h;
        } else {
            fp = seq_base<X>(a.f, pair, N); gp = seq_base<X>(a.g, pair, N);
            hp = X::GARNER ? nullptr : a.h + (size_t)pair * N;
        }
    };
    constexpr uint32_t INB = X::IN64 ? 8u : (uint32_t)sizeof(W);     // bytes per input element
    for (long long rho = base + gid; rho < a.nrows; rho += stride) {
        const W *fp, *gp;
        W *hp;
        ptrs(rho, fp, gp, hp);
        if (tau == 0 && rho + stride < a.nrows) {
            const W *fn, *gn;
            W *hn;
            ptrs(rho + stride, fn, gn, hn);
            prefetch_l2(fn, N * INB);
            prefetch_l2(gn, N * INB);
        }
        W v[2][R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            v[0][k] = ld_elem<X>(fp, b0 + ((uint32_t)k << lo0), xa);
            v[1][k] = ld_elem<X>(gp, b0 + ((uint32_t)k << lo0), xa);
        }
        fwd_all<W, L, L, 0, 2, TW_SMEM, true>(v, 0u, tau, S, gid, stw, a.c);
#pragma unroll
        for (int k = 0; k < R; ++k) v[0][k] = pointwise(v[0][k], v[1][k], a.c);
        dit_all<W, L, last, TW_SMEM>(v[0], 0u, tau, S, gid, stw, a.c);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const uint32_t x = b0 + ((uint32_t)k << lo0);
            st_out<X>(hp, a.pair0 + rho, N, (N - x) & (N - 1u), canon<W>(v[0][k], (W)1, a.c.onep, a.c.m), xa);
        }
    }
}

template <typename W, int L, int SRC, int BLK = BLOCK>
__global__ void __launch_bounds__(BLK, BLOCK / BLK) k_conv_fused(const __grid_constant__ RowArgs<W> a)
{
    constexpr int GPC = RowShape<W, L, L, BLK>::GPC;
    conv_fused_body<W, L, SRC>(a, (long long)blockIdx.x * GPC, (long long)gridDim.x * GPC);
}

// ---- column/row fused kernel ---------------------------------------------
//
// For 2^RW < N <= 2^LR_max (RW = log2 of the 32 x R elements one warp holds:
// 10 for 32-bit words), the index splits into LC = L - RW top bits and RW low
// bits.  The forward tree's first LC levels act on "columns" (fixed low bits,
// 2^LC elements each): each thread holds whole columns in registers, whose
// node twiddles are the first 2^LC - 1 table entries for every column.  One
// block-wide transpose through shared memory then gives every warp a
// contiguous "row" of 2^RW elements, whose remaining levels (and the first
// RW levels of the inverse) need only warp-level exchanges, so warps run
// independently and one warp's exchanges overlap another's arithmetic.  The
// inverse's last LC levels act on columns again; their twiddles are the runs
// z_{brv_RW(c) 2^J + t}.  Shared memory holds, per row, the f and g slices
// side by side (stride ROWP of the row geometry).

// Forward node levels of one column of RC = 2^LC elements stored at v[OFF ..].
// The column's top bit sits at global level DG0 (0 when the columns hold the
// top bits of the whole transform); node indices at the level of register
// bit J are nbase_J + (k >> (J + 1)), with nbase_J = rowbase >> (J + 1) for
// a row that is itself part of a longer transform (rowbase = its global
// index offset divided by 2^RW).
template <typename W, int LC, int OFF, int J, int DG0, int TWS, int RR>
__device__ __forceinline__ void colf_levels(W (&v)[RR], uint32_t rowbase, const W *__restrict__ tw, const ModC<W> &c)
{
    if constexpr (J >= 0) {
        constexpr int RC = 1 << LC;
        constexpr int dg = DG0 + LC - 1 - J;
        if constexpr (dg == 0) {
#pragma unroll
            for (int k = 0; k < RC; ++k) {
                if (k & (1 << J)) continue;
                ct_bfly_one<W>(v[OFF + k], v[OFF + (k | (1 << J))], c);
            }
        } else {
            constexpr int CNT = RC >> (J + 1);
            constexpr int CH = (CNT >= 2 && tw_per_chunk<W>() == 2) ? 2 : 1;
            const uint32_t nbase = rowbase >> (J + 1);
#pragma unroll
            for (int t0 = 0; t0 < CNT; t0 += CH) {
                W z[CH], zp[CH];
                load_tw<W, CH, TWS>(tw, nbase, (uint32_t)t0, z, zp);
#pragma unroll
                for (int tt = 0; tt < CH; ++tt)
#pragma unroll
                    for (int j = 0; j < (1 << J); ++j) {
                        const int k = ((t0 + tt) << (J + 1)) | j;
                        // whole sequence: node 0 has the twiddle 1 (bound note at fwd_level)
                        if (DG0 == 0 && dg <= 4 && t0 + tt == 0) ct_bfly_unit<W>(v[OFF + k], v[OFF + (k | (1 << J))], c.m << dg);
                        else ct_bfly<W>(v[OFF + k], v[OFF + (k | (1 << J))], z[tt], zp[tt], c);
                    }
            }
        }
        colf_levels<W, LC, OFF, J - 1, DG0, TWS, RR>(v, rowbase, tw, c);
    }
}

// Transposed (inverse-direction) node levels of one column, deepest first:
// the exact reverse of colf_levels with the same twiddles.  Inputs < 2m,
// outputs < 2m.
template <typename W, int LC, int OFF, int J, int DG0, int TWS, int RR>
__device__ __forceinline__ void colg_levels(W (&v)[RR], uint32_t rowbase, const W *__restrict__ tw, const ModC<W> &c)
{
    if constexpr (J < LC) {
        constexpr int RC = 1 << LC;
        constexpr int dg = DG0 + LC - 1 - J;
        if constexpr (dg == 0) {
#pragma unroll
            for (int k = 0; k < RC; ++k) {
                if (k & (1 << J)) continue;
                gs_bfly_one<W>(v[OFF + k], v[OFF + (k | (1 << J))], c);
            }
        } else {
            constexpr int CNT = RC >> (J + 1);
            constexpr int CH = (CNT >= 2 && tw_per_chunk<W>() == 2) ? 2 : 1;
            const uint32_t nbase = rowbase >> (J + 1);
#pragma unroll
            for (int t0 = 0; t0 < CNT; t0 += CH) {
                W z[CH], zp[CH];
                load_tw<W, CH, TWS>(tw, nbase, (uint32_t)t0, z, zp);
#pragma unroll
                for (int tt = 0; tt < CH; ++tt)
#pragma unroll
                    for (int j = 0; j < (1 << J); ++j) {
                        const int k = ((t0 + tt) << (J + 1)) | j;
                        gs_bfly<W>(v[OFF + k], v[OFF + (k | (1 << J))], z[tt], zp[tt], c);
                    }
            }
        }
        colg_levels<W, LC, OFF, J + 1, DG0, TWS, RR>(v, rowbase, tw, c);
    }
}

template <typename W, int LC, int JC, int CPT, int DG0, int TWS, int RR>
__device__ __forceinline__ void colg_all(W (&v)[RR], uint32_t rowbase, const W *__restrict__ tw, const ModC<W> &c)
{
    if constexpr (JC < CPT) {
        colg_levels<W, LC, JC * (1 << LC), 0, DG0, TWS, RR>(v, rowbase, tw, c);
        colg_all<W, LC, JC + 1, CPT, DG0, TWS, RR>(v, rowbase, tw, c);
    }
}

// Inverse (decimation-in-time) levels l = RW + J of one column c, tlo = brv_RW(c).
template <typename W, int LC, int OFF, int J, int TWS, int RR>
__device__ __forceinline__ void cold_levels(W (&v)[RR], uint32_t tlo, const W *__restrict__ tw, const ModC<W> &c)
{
    if constexpr (J < LC) {
        constexpr int RC = 1 << LC;
        constexpr int CNT = 1 << J;
        constexpr int CH = (CNT >= 2 && tw_per_chunk<W>() == 2) ? 2 : 1;
        const uint32_t run = tlo << J;
#pragma unroll
        for (int t0 = 0; t0 < CNT; t0 += CH) {
            W z[CH], zp[CH];
            load_tw<W, CH, TWS>(tw, run, (uint32_t)t0, z, zp);
#pragma unroll
            for (int tt = 0; tt < CH; ++tt) {
                const int j = brv_c<J>(t0 + tt);
#pragma unroll
                for (int hi = 0; hi < (RC >> (J + 1)); ++hi) {
                    const int k = (hi << (J + 1)) | j;
                    ct_bfly<W>(v[OFF + k], v[OFF + (k | (1 << J))], z[tt], zp[tt], c);
                }
            }
        }
        cold_levels<W, LC, OFF, J + 1, TWS, RR>(v, tlo, tw, c);
    }
}

// All columns JC .. CPT-1 held by a thread (column j at v[j * 2^LC ..]).
template <typename W, int LC, int JC, int CPT, int DG0, int TWS, int RR>
__device__ __forceinline__ void colf_all(W (&v)[RR], uint32_t rowbase, const W *__restrict__ tw, const ModC<W> &c)
{
    if constexpr (JC < CPT) {
        colf_levels<W, LC, JC * (1 << LC), LC - 1, DG0, TWS, RR>(v, rowbase, tw, c);
        colf_all<W, LC, JC + 1, CPT, DG0, TWS, RR>(v, rowbase, tw, c);
    }
}

template <typename W, int LC, int RW, int JC, int CPT, int TPP, int TWS, int RR>
__device__ __forceinline__ void cold_all(W (&v)[RR], uint32_t ptau, const W *__restrict__ tw, const ModC<W> &c)
{
    if constexpr (JC < CPT) {
        const uint32_t col = ptau + (uint32_t)JC * TPP;
        cold_levels<W, LC, JC * (1 << LC), 0, TWS, RR>(v, __brev(col) >> (32 - RW), tw, c);
        cold_all<W, LC, RW, JC + 1, CPT, TPP, TWS, RR>(v, ptau, tw, c);
    }
}

template <typename W, int L, int LROW = L, int BLK = BLOCK>
struct CRShape {
    static constexpr int RW = Arith<W>::RB + 5;
    static constexpr int LC = LROW - RW;                    // column bits inside one row
    static constexpr int RC = 1 << LC;
    using GR = Geo<W, RW>;
    static constexpr int TPP = 32 * RC;                     // threads per row
    static constexpr int PPC = BLK / TPP;                   // rows per block
    static_assert(PPC >= 1, "a row needs more threads than the block has");
    static constexpr int CPT = (1 << RW) / TPP;             // columns per thread
    // shared twiddles: the whole table (whole sequences) or only the entries
    // below 2^(LROW-1) that the inverse levels inside a row read (split rows)
    static constexpr int TWL = (L == LROW) ? L : 0;         // split rows read the plan's table
    static constexpr size_t smem = TwBytes<W, TWL>::v + (size_t)PPC * RC * 2 * GR::ROWP * sizeof(W);
};

// Column/row fused convolution.  L == LROW: whole sequences (f, g, h or the
// descriptor list; output canonical at <-x>_N).  L > LROW: one row of 2^LROW
// elements of the split path per row group, inputs F~, G~ and output H~ in
// the wave's scratch; the forward node twiddles of such a row depend on the
// row and are read from the plan's table, the inverse ones do not and are
// read from shared memory.
// Rows [base + row group, end) by steps of stride; end is a.nrows unless ITEM.
// OUT 0: canonical at <-x>_N (a whole convolution); OUT 1: lazy residues in
// natural order (a row of a convolution's split path, after the twist).
template <typename W, int L, int LROW, int SRC, bool ITEM = false, int OUT = 0, class X = NoExact, int BLK = BLOCK>
__device__ __forceinline__ void conv_cr_body(const RowArgs<W> &a, long long base, long long stride, long long end = 0,
                                             const ExactArgs *xa = nullptr)
{
    using SH = CRShape<W, L, LROW, BLK>;
    using GR = typename SH::GR;
    constexpr int RW = SH::RW, LC = SH::LC, RC = SH::RC, TPP = SH::TPP, PPC = SH::PPC, CPT = SH::CPT;
    constexpr int R = GR::R;
    static_assert(LC >= 1 && CPT * RC == R, "column/row split");
    constexpr bool FULL = (L == LROW);
    constexpr int FTW = FULL ? TW_SMEM : TW_GLOBAL;         // forward twiddle source
    constexpr uint32_t N = 1u << L;
    constexpr int last = GR::NPASS - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int pid = threadIdx.x / TPP;
    const uint32_t ptau = threadIdx.x % TPP;
    const int wr = (int)(ptau >> 5);
    const uint32_t lane = ptau & 31u;
    W *stw = reinterpret_cast<W *>(smem_raw);
    W *P = reinterpret_cast<W *>(smem_raw + TwBytes<W, SH::TWL>::v) + (size_t)pid * RC * 2 * GR::ROWP;
    W *Srow = P + (size_t)wr * 2 * GR::ROWP;                // this warp's g slice (also H); f slice follows
    const W *ftw = FULL ? stw : a.tw;
    const uint32_t b0 = GR::base(0, lane);
    constexpr int lo0 = GR::lo(0);
    if constexpr (FULL) {
        stage_twiddles<W>(a.tw, stw, TwBytes<W, SH::TWL>::pairs);
        __syncthreads();
    }

    // The row groups of a block synchronise block-wide and step through the
    // rows in rounds together (a group whose row of the round is past the
    // end skips its memory accesses), so every group runs the same phase at
    // the same time: measured 9% (2^11) and 15% (2^12) faster than a
    // barrier per group, whose groups drift apart across the unrolled code.
    auto psync = [&]() { __syncthreads(); };
    auto ptrs = [&](long long rho, const W *&fp, const W *&gp, W *&hp, uint32_t &rowoff) {
        if constexpr (FULL) {
            const long long pair = a.pair0 + rho;
            if constexpr (SRC == 1) {
                const DevDesc<W> d = a.descs[pair];
                fp = d.f; gp = d.g; hp = d.h;
            } else {
                fp = seq_base<X>(a.f, pair, N); gp = seq_base<X>(a.g, pair, N);
                hp = X::GARNER ? nullptr : a.h + (size_t)pair * N;
            }
            rowoff = 0;
        } else {
            const long long pw = rho >> (L - LROW);
            const uint32_t row = (uint32_t)rho & ((1u << (L - LROW)) - 1u);
            const size_t off = (size_t)pw * N + ((size_t)row << LROW);
            fp = a.f + off; gp = a.g + off; hp = a.h + off;
            rowoff = row << LROW;
        }
    };
    // v[1] carries this row's f, loaded during the previous row's inverse
    // phases (the registers are free after the pointwise product); g is
    // loaded into v[0] while f's column levels run.  (Staging g in the idle
    // g slices with cp.async instead was measured slower: the extra shared
    // memory traffic costs more than the latency it hides.)
    auto load_cols = [&](const W *src, W (&dst)[R]) {
#pragma unroll
        for (int j = 0; j < CPT; ++j)
#pragma unroll
            for (int k = 0; k < RC; ++k) dst[j * RC + k] = ld_elem<X>(src, ptau + (uint32_t)j * TPP + ((uint32_t)k << RW), xa);
    };
    constexpr uint32_t INB = X::IN64 ? 8u : (uint32_t)sizeof(W);     // bytes per input element
    const long long lim = ITEM ? end : a.nrows;
    W v[2][R];
    const W *fp = nullptr, *gp = nullptr;
    W *hp = nullptr;
    uint32_t rowoff = 0;
    // (split rows keep no prefetched registers across their inverse: it reads
    // its twiddles from global memory and needs the registers itself)
    constexpr bool PREF = FULL;
    if (PREF && base + pid < lim) {
        ptrs(base + pid, fp, gp, hp, rowoff);
        load_cols(fp, v[1]);
    }
    for (long long round = base; round < lim; round += stride) {
        const long long rho = round + pid;
        const bool live = PPC == 1 || rho < lim;            // this group's row of the round exists
        if (!PREF && live) {
            ptrs(rho, fp, gp, hp, rowoff);
            load_cols(fp, v[1]);
        }
        W *const hcur = hp;
        const uint32_t rcur = live ? rowoff : 0u;
        const W *gcur = gp;
        if (ptau == 0 && rho + stride < lim) {
            const W *fn, *gn;
            W *hn;
            uint32_t ro;
            ptrs(rho + stride, fn, gn, hn, ro);
            prefetch_l2(fn, (1u << LROW) * INB);
            prefetch_l2(gn, (1u << LROW) * INB);
        }
        // forward, column phase: columns c = ptau + j TPP, elements x = c + k 2^RW.
        // No barrier before the column stores: the f slices were last read in
        // the previous row's row phase, before the last barrier, and in the g
        // slices every thread writes only the positions of its own columns,
        // which it alone read in the previous row's inverse column phase.
        // (Measured on GB300 at 4096 x 2^14: moving the barrier that stood
        // before both stores to after f's made the kernel 2.9% faster,
        // removing it 0.8% more.)
        if (live) load_cols(gcur, v[0]);
        colf_all<W, LC, 0, CPT, L - LROW, FTW, R>(v[1], rcur >> RW, ftw, a.c);
#pragma unroll
        for (int j = 0; j < CPT; ++j)
#pragma unroll
            for (int k = 0; k < RC; ++k) {
                const uint32_t y = ptau + (uint32_t)j * TPP;
                P[(size_t)k * 2 * GR::ROWP + GR::ROWP + GR::pad(y)] = v[1][j * RC + k];   // f
            }
        colf_all<W, LC, 0, CPT, L - LROW, FTW, R>(v[0], rcur >> RW, ftw, a.c);
#pragma unroll
        for (int j = 0; j < CPT; ++j)
#pragma unroll
            for (int k = 0; k < RC; ++k) {
                const uint32_t y = ptau + (uint32_t)j * TPP;
                P[(size_t)k * 2 * GR::ROWP + GR::pad(y)] = v[0][j * RC + k];              // g
            }
        psync();
        // forward, row phase (warp wr owns row wr of this row group)
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const uint32_t y = b0 + ((uint32_t)k << lo0);
            v[0][k] = Srow[GR::pad(y)];
            v[1][k] = Srow[GR::ROWP + GR::pad(y)];
        }
        fwd_all<W, L, RW, 0, 2, FTW>(v, rcur + ((uint32_t)wr << RW), lane, Srow, 0, ftw, a.c);
#pragma unroll
        for (int k = 0; k < R; ++k) v[0][k] = pointwise(v[1][k], v[0][k], a.c);
        if (PREF && rho + stride < lim) {
            ptrs(rho + stride, fp, gp, hp, rowoff);
            load_cols(fp, v[1]);                            // next row's f
        }
        // inverse, row phase: decimation in time for whole sequences; for a
        // row of the split path the transposed tree, whose twiddles (like the
        // forward ones) are contiguous runs of the plan's table
        if constexpr (FULL) dit_all<W, RW, last, TW_SMEM>(v[0], (uint32_t)wr << RW, lane, Srow, 0, stw, a.c);
        else inv_all<W, L, RW, last, TW_GLOBAL>(v[0], rcur + ((uint32_t)wr << RW), lane, Srow, 0, a.tw, a.c);
#pragma unroll
        for (int k = 0; k < R; ++k) Srow[GR::pad(b0 + ((uint32_t)k << lo0))] = v[0][k];
        psync();
        // inverse, column phase
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const uint32_t col = ptau + (uint32_t)j * TPP;
#pragma unroll
            for (int k = 0; k < RC; ++k) v[0][j * RC + k] = P[(size_t)k * 2 * GR::ROWP + GR::pad(col)];
        }
        if constexpr (FULL) cold_all<W, LC, RW, 0, CPT, TPP, TW_SMEM, R>(v[0], ptau, stw, a.c);
        else colg_all<W, LC, 0, CPT, L - LROW, TW_GLOBAL, R>(v[0], rcur >> RW, a.tw, a.c);
        if (!live) continue;                                // (no barrier follows in this round)
#pragma unroll
        for (int j = 0; j < CPT; ++j)
#pragma unroll
            for (int k = 0; k < RC; ++k) {
                const uint32_t x = ptau + (uint32_t)j * TPP + ((uint32_t)k << RW);
                if constexpr (FULL && OUT == 0)
                    st_out<X>(hcur, a.pair0 + rho, N, (N - x) & (N - 1u), canon<W>(v[0][j * RC + k], (W)1, a.c.onep, a.c.m), xa);
                else hcur[x] = v[0][j * RC + k];
            }
    }
}

template <typename W, int L, int LROW, int SRC, int OUT = 0, int BLK = BLOCK>
__global__ void __launch_bounds__(BLK, BLOCK / BLK) k_conv_cr(const __grid_constant__ RowArgs<W> a)
{
    constexpr int PPC = CRShape<W, L, LROW, BLK>::PPC;
    conv_cr_body<W, L, LROW, SRC, false, OUT, NoExact, BLK>(a, (long long)blockIdx.x * PPC, (long long)gridDim.x * PPC);
}

// The exact convolution's fused launches (whole sequences, contiguous):
// X = ExactResidues for every prime but the last (its residues of h go to
// a.h), X = ExactGarner for the last (h goes to e.h64 as signed integers).
template <typename W, int L, class X>
__global__ void __launch_bounds__(BLOCK, 1) k_conv_exact(const __grid_constant__ RowArgs<W> a,
                                                          const __grid_constant__ ExactArgs e)
{
    constexpr int RW = Arith<W>::RB + 5;
    if constexpr (L <= RW) {
        constexpr int GPC = RowShape<W, L, L>::GPC;
        conv_fused_body<W, L, 0, X>(a, (long long)blockIdx.x * GPC, (long long)gridDim.x * GPC, &e);
    } else {
        constexpr int PPC = CRShape<W, L, L>::PPC;
        conv_cr_body<W, L, L, 0, false, 0, X>(a, (long long)blockIdx.x * PPC, (long long)gridDim.x * PPC, 0, &e);
    }
}

// ---- one persistent launch for every whole-sequence length of a batch ----
//
// Work items {log2 N, first pair, count} of a batch plan's descriptor list
// (grouped by length) are pulled by the blocks with an atomic counter; a
// block runs the item with the fused body of its length, staging that
// length's twiddle table into shared memory first.  Blocks never wait on
// one another.

struct WorkItem {
    int L;
    int reserved;
    long long first;
    long long count;
};

// The per-length arguments (descriptor list, twiddle table, constants) travel
// by value in the kernel's parameter space, so each length's body reads them
// as constant-bank operands, as the single-length kernels do, instead of
// holding them in registers.
template <typename W> struct PersistArgs {
    const WorkItem *items;
    int nitems;
    int *counter;                      // zeroed before each launch
    RowArgs<W> cls[LRMax<W>::v + 1];   // indexed by log2 N
};

template <typename W, int L>
__device__ __forceinline__ void persist_item(const PersistArgs<W> &a, const WorkItem &w)
{
    constexpr int RW = Arith<W>::RB + 5;
    // rows [first, first + count) of the descriptor list; the one-warp body
    // takes them as a local copy of its arguments with nrows set (it compiles
    // without spills that way), the column/row body as an explicit bound
    if constexpr (L <= RW) {
        RowArgs<W> ra = a.cls[L];
        ra.nrows = w.first + w.count;
        conv_fused_body<W, L, 1>(ra, w.first, RowShape<W, L, L>::GPC);
    }
    else conv_cr_body<W, L, L, 1, true>(a.cls[L], w.first, CRShape<W, L, L>::PPC, w.first + w.count);
}

template <typename W, int L, int HI>
__device__ __forceinline__ void persist_dispatch(const PersistArgs<W> &a, const WorkItem &w)
{
    if constexpr (L <= HI) {
        if (w.L == L) persist_item<W, L>(a, w);
        else persist_dispatch<W, L + 1, HI>(a, w);
    }
}

// HI: the longest length the kernel is compiled for (the one-warp lengths
// only, or every whole-sequence length).
template <typename W, int HI>
__global__ void __launch_bounds__(BLOCK, 1) k_conv_persistent(const __grid_constant__ PersistArgs<W> a)
{
    __shared__ int item;
    for (;;) {
        __syncthreads();                                   // previous item done with shared memory
        if (threadIdx.x == 0) item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int it = item;
        if (it >= a.nitems) break;
        persist_dispatch<W, 0, HI>(a, a.items[it]);
    }
}

// Natural-order forward transform (Eq. 2) or inverse transform (Eq. 3) of
// whole sequences (L <= LR_max).  The forward tree leaves X(brv(x)) at x; a
// shared-memory pass puts it back in natural order.  The inverse is
// N^-1 R F: same forward tree, output index <-u>_N, factor N^-1.
template <typename W> struct NttArgs {
    const W *x;
    W *y;
    long long batch;
    const W *tw;
    ModC<W> c;
};

template <typename W, int L, bool INV>
__global__ void __launch_bounds__(BLOCK, 1) k_ntt_rows(const __grid_constant__ NttArgs<W> a)
{
    using G = Geo<W, L>;
    constexpr int T = G::T, R = G::R, GPC = RowShape<W, L, L>::GPC;
    constexpr uint32_t N = 1u << L;
    constexpr int last = G::NPASS - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gid = threadIdx.x / T;
    const uint32_t tau = threadIdx.x % T;
    W *stw = reinterpret_cast<W *>(smem_raw);
    W *S = reinterpret_cast<W *>(smem_raw + TwBytes<W, L>::v) + (size_t)gid * G::ROWP;
    const uint32_t b0 = G::base(0, tau), bl = G::base(last, tau);
    constexpr int lo0 = G::lo(0), lol = G::lo(last);
    stage_twiddles<W>(a.tw, stw, TwBytes<W, L>::pairs);
    __syncthreads();
    const W scale = INV ? a.c.ninv : (W)1;
    const W scalep = INV ? a.c.ninvp : a.c.onep;

    // 32-bit words: the next sequence is loaded into w while this one is
    // transformed (every group of a block otherwise waits on its loads at
    // the same time); 64-bit words have no registers to spare for it
    constexpr bool PF = sizeof(W) == 4;
    const long long step = (long long)gridDim.x * GPC;
    long long rho = (long long)blockIdx.x * GPC + gid;
    W v[1][R], w[R];
    auto load = [&](long long r, W (&dst)[R]) {
        const W *xp = a.x + (size_t)r * N;
#pragma unroll
        for (int k = 0; k < R; ++k) dst[k] = xp[b0 + ((uint32_t)k << lo0)];
    };
    if (PF && rho < a.batch) load(rho, v[0]);
    for (; rho < a.batch; rho += step) {
        W *yp = a.y + (size_t)rho * N;
        if (!PF) load(rho, v[0]);
        const bool more = PF && rho + step < a.batch;
        if (more) load(rho + step, w);
        fwd_all<W, L, L, 0, 1, TW_SMEM>(v, 0u, tau, S, gid, stw, a.c);
        group_sync<T>(gid);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const uint32_t x = bl + ((uint32_t)k << lol);
            const uint32_t u = L == 0 ? 0u : (__brev(x) >> (32 - L));
            S[G::pad(u)] = v[0][k];
        }
        group_sync<T>(gid);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            // output index t (a warp's stores are one aligned run); the
            // inverse takes its value from <-t>_N
            const uint32_t t = b0 + ((uint32_t)k << lo0);
            const uint32_t u = INV ? ((N - t) & (N - 1u)) : t;
            yp[t] = csub<W>(shoup<W>(S[G::pad(u)], scale, scalep, a.c.m), a.c.m);
        }
        if (more) {
#pragma unroll
            for (int k = 0; k < R; ++k) v[0][k] = w[k];
        }
    }
}

// Split path for L > LR: "column" transforms of the top LC = L - LR index
// bits.  Element (c, k) of a sequence is x = c + k 2^LR (c < 2^LR, k < 2^LC);
// every level of the top bits has node index k >> (bits below), the same for
// all columns.  NS sequences per thread (f and g).
template <typename W> struct ColArgs {
    const W *src0;      // SRC == 0: contiguous batch base of sequence 0 (f)
    const W *src1;      // ... of sequence 1 (g)
    const DevDesc<W> *descs;   // SRC == 1
    W *dst0;            // scratch of the wave (F~), [pairs][N]
    W *dst1;            // scratch (G~)
    W *out;             // cols_inv, DST == 0: contiguous output base
    long long npairs;   // pairs in this wave
    long long pair0;    // first pair of the wave in the batch / descriptor list
    const W *tw;
    ModC<W> c;
    const W *pw;        // convolutions: (w^e, Shoup quotient) pairs, e < N (the twist)
    const W *pwl;       // (w^(s l), quotient) at s 32 + l, s < 2^(L-LR), l < 32
    const W *pd;        // one column pass: (w^(brv(k) t), quotient) at x = t + k 2^LR
};

// The four-step twist, one of the two forms of the split path of
// convolutions and natural-order transforms (the plan picks one per word
// size and length; the autotuner measures both).  In the other form the rows
// read their node twiddles, which then depend on the row, from the plan's
// table.  With the twist: after the column levels, element (r, t) -- r the
// top L - LR index bits at their tree position, t the low LR bits -- is
// multiplied by w^(brv(r) t).  That turns every row's remaining levels into
// the length-2^LR transform with the uniform table z'_i = w'^brv(i),
// w' = w^(2^(L-LR)), whose entries are the first 2^(LR-1) of the plan's
// table; the rows then run the whole-sequence convolution kernel (or, for
// transforms, k_rows_uni).  The inverse (the transposed tree) applies the
// same diagonal between the rows and the transposed column levels.  Output
// in [0, 2m).
//
// With one column pass the factor of element x = t + k 2^LR depends on x
// alone (not on the pair), so the plan stores it at x (ColArgs::pd): one
// coalesced, L2-resident vector load and one Shoup product per element.
// With two column passes (k_cols_mid_*) it is split as w^(s t0) w^(s l),
// t = t0 + l, l = t mod 32 (the lane): the first is the same for a warp (one
// broadcast load), the second comes from a small lane table (s, l) ->
// w^(s l), coalesced; two Shoup products.  Each (power, Shoup quotient)
// pair is one vector load.
template <typename W> struct PairVec;
template <> struct PairVec<uint32_t> { using T = uint2; };
template <> struct PairVec<uint64_t> { using T = ulonglong2; };

template <typename W>
__device__ __forceinline__ void ld_pair_g(const W *p, W &z, W &zp)
{
    const typename PairVec<W>::T q = __ldg(reinterpret_cast<const typename PairVec<W>::T *>(p));
    z = q.x; zp = q.y;
}

template <typename W>
__device__ __forceinline__ void ld_pair(const W *p, W &z, W &zp)
{
    const typename PairVec<W>::T q = *reinterpret_cast<const typename PairVec<W>::T *>(p);
    z = q.x; zp = q.y;
}

// The twist factor of (s, t): e = s (t - l) mod N for the warp-uniform part;
// lt is the lane table (shared memory, or the plan's copy).
template <typename W, int L>
__device__ __forceinline__ void twist_factors(uint32_t s, uint32_t t, const ColArgs<W> &a, const W *lt, W &z0, W &z0p,
                                              W &z1, W &z1p)
{
    const uint32_t l = t & 31u;
    const uint32_t e = (s * (t - l)) & ((1u << L) - 1u);
    ld_pair_g<W>(a.pw + 2 * (size_t)e, z0, z0p);
    ld_pair<W>(lt + 2 * ((size_t)s * 32 + l), z1, z1p);
}

template <typename W, int L>
__device__ __forceinline__ W twist(W v, uint32_t s, uint32_t t, const ColArgs<W> &a, const W *lt)
{
    W z0, z0p, z1, z1p;
    twist_factors<W, L>(s, t, a, lt, z0, z0p, z1, z1p);
    return shoup<W>(shoup<W>(v, z1, z1p, a.c.m), z0, z0p, a.c.m);
}

template <int BITS>
__host__ __device__ constexpr uint32_t brv_c32(uint32_t k)
{
    uint32_t r = 0;
    for (int i = 0; i < BITS; ++i) r |= ((k >> i) & 1u) << (BITS - 1 - i);
    return r;
}

// Pairs 0 .. CNT-1 of the plan's table (the same for every column).
template <typename W, int CNT>
__device__ __forceinline__ void load_tw_run(const W *__restrict__ tw, W (&z)[CNT], W (&zp)[CNT])
{
#pragma unroll
    for (int t = 0; t < CNT; ++t) {
        W a[1], ap[1];
        load_tw<W, 1, TW_GLOBAL>(tw, 0u, (uint32_t)t, a, ap);
        z[t] = a[0]; zp[t] = ap[0];
    }
}

template <typename W, int L, int LR, int J>
__device__ __forceinline__ void col_fwd_level(W (&v)[1 << (L - LR)], const W *__restrict__ tw, const ModC<W> &c)
{
    // J = register bit, element bit b = LR + J, global level L - 1 - b
    constexpr int RC = 1 << (L - LR);
    constexpr int dg = L - LR - 1 - J;
    if constexpr (dg == 0) {
#pragma unroll
        for (int k = 0; k < RC; ++k) {
            if (k & (1 << J)) continue;
            ct_bfly_one<W>(v[k], v[k | (1 << J)], c);
        }
    } else {
        constexpr int CNT = RC >> (J + 1);
        W z[CNT], zp[CNT];
        load_tw_run<W, CNT>(tw, z, zp);
#pragma unroll
        for (int k = 0; k < RC; ++k) {
            if (k & (1 << J)) continue;
            ct_bfly<W>(v[k], v[k | (1 << J)], z[k >> (J + 1)], zp[k >> (J + 1)], c);
        }
    }
}

template <typename W, int L, int LR, int J>
__device__ __forceinline__ void col_fwd_levels(W (&v)[1 << (L - LR)], const W *__restrict__ tw, const ModC<W> &c)
{
    if constexpr (J >= 0) {
        col_fwd_level<W, L, LR, J>(v, tw, c);
        col_fwd_levels<W, L, LR, J - 1>(v, tw, c);
    }
}

// (the twisted 32-bit form holds f and g at once: at most 80 registers keep
// three blocks, 24 warps, on an SM for the loads in flight)
template <typename W, int L, int LR, int NS, int SRC, bool TWIST>
__global__ void __launch_bounds__(256, (TWIST && NS == 2 && sizeof(W) == 4) ? 3 : 1)
    k_cols_fwd(const __grid_constant__ ColArgs<W> a)
{
    constexpr int RC = 1 << (L - LR);
    constexpr uint32_t N = 1u << L;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.npairs << LR) return;
    const long long pw = idx >> LR;
    const uint32_t col = (uint32_t)idx & ((1u << LR) - 1u);
    auto source = [&](int s) -> const W * {
        if constexpr (SRC == 1) {
            const DevDesc<W> d = a.descs[a.pair0 + pw];
            return s == 0 ? d.f : d.g;
        } else {
            return (s == 0 ? a.src0 : a.src1) + (size_t)(a.pair0 + pw) * N;
        }
    };
    if constexpr (TWIST && NS == 2 && sizeof(W) == 4) {
        // 32-bit words: f and g together, so that each twist factor is
        // loaded once for both
        const W *sf = source(0), *sg = source(1);
        W vf[RC], vg[RC];
#pragma unroll
        for (int k = 0; k < RC; ++k) {
            vf[k] = sf[col + ((uint32_t)k << LR)];
            vg[k] = sg[col + ((uint32_t)k << LR)];
        }
        col_fwd_levels<W, L, LR, L - LR - 1>(vf, a.tw, a.c);
        col_fwd_levels<W, L, LR, L - LR - 1>(vg, a.tw, a.c);
        W *df = a.dst0 + (size_t)pw * N, *dg = a.dst1 + (size_t)pw * N;
#pragma unroll
        for (int k = 0; k < RC; ++k) {
            const uint32_t x = col + ((uint32_t)k << LR);
            W z, zp;
            ld_pair_g<W>(a.pd + 2 * (size_t)x, z, zp);
            df[x] = csub<W>(shoup<W>(vf[k], z, zp, a.c.m), a.c.m);
            dg[x] = csub<W>(shoup<W>(vg[k], z, zp, a.c.m), a.c.m);
        }
    } else {
#pragma unroll 1
        for (int s = 0; s < NS; ++s) {
            const W *src = source(s);
            W *dst = (s == 0 ? a.dst0 : a.dst1) + (size_t)pw * N;
            W v[RC];
#pragma unroll
            for (int k = 0; k < RC; ++k) v[k] = src[col + ((uint32_t)k << LR)];
            col_fwd_levels<W, L, LR, L - LR - 1>(v, a.tw, a.c);
            if constexpr (TWIST) {
#pragma unroll
                for (int k = 0; k < RC; ++k) {
                    W z, zp;
                    ld_pair_g<W>(a.pd + 2 * (size_t)(col + ((uint32_t)k << LR)), z, zp);
                    v[k] = csub<W>(shoup<W>(v[k], z, zp, a.c.m), a.c.m);
                    // 64-bit words: keep the compiler from hoisting every table
                    // load ahead of the products (it spills them otherwise)
                    if constexpr (sizeof(W) == 8 && RC > 8)
                        if ((k & 7) == 7) asm volatile("" ::: "memory");
                }
            }
#pragma unroll
            for (int k = 0; k < RC; ++k) dst[col + ((uint32_t)k << LR)] = v[k];
        }
    }
}

// Transposed top levels of the split path on column c (elements
// x = c + k 2^LR): node twiddles k >> (J + 1), the same for every column.
// Inputs < 2m; then the output stage: index <-x>_N, canonical residue.
// DST 0: contiguous out; 1: descriptor h.
template <typename W, int L, int LR, int DST, bool TWIST>
__device__ __forceinline__ void cols_inv_body(const ColArgs<W> &a)
{
    constexpr int LC = L - LR, RC = 1 << LC;
    constexpr uint32_t N = 1u << L;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.npairs << LR) return;
    const long long pw = idx >> LR;
    const uint32_t col = (uint32_t)idx & ((1u << LR) - 1u);
    const W *src = a.dst0 + (size_t)pw * N;
    W *out;
    if constexpr (DST == 1) out = a.descs[a.pair0 + pw].h;
    else out = a.out + (size_t)(a.pair0 + pw) * N;
    W v[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) v[k] = src[col + ((uint32_t)k << LR)];
    if constexpr (TWIST) {
#pragma unroll
        for (int k = 0; k < RC; ++k) {
            W z, zp;
            ld_pair_g<W>(a.pd + 2 * (size_t)(col + ((uint32_t)k << LR)), z, zp);
            v[k] = shoup<W>(v[k], z, zp, a.c.m);
            if constexpr (sizeof(W) == 8 && RC > 8)
                if ((k & 7) == 7) asm volatile("" ::: "memory");
        }
    }
    colg_levels<W, LC, 0, 0, 0, TW_GLOBAL, RC>(v, 0u, a.tw, a.c);
#pragma unroll
    for (int k = 0; k < RC; ++k) {
        const uint32_t x = col + ((uint32_t)k << LR);
        out[(N - x) & (N - 1u)] = csub<W>(v[k], a.c.m);
    }
}

template <typename W, int L, int LR, int DST, bool TWIST>
__global__ void __launch_bounds__(256) k_cols_inv(const __grid_constant__ ColArgs<W> a)
{
    cols_inv_body<W, L, LR, DST, TWIST>(a);
}

// The same with at most 48 registers, five blocks per SM for the loads in
// flight: used for 32-bit words with five column bits, where the plain bound
// takes 56 registers with contiguous output and 58 with descriptor output
// (four blocks); measured on GB300 1.7% faster for 64 x 2^19 (contiguous)
// and 12-14% faster for 714 x 2^19 (descriptors).  (An explicit bound raises
// the register count of the shorter and 64-bit forms instead, so they keep
// the plain one.)
template <typename W, int L, int LR, int DST, bool TWIST>
__global__ void __launch_bounds__(256, 5) k_cols_inv5(const __grid_constant__ ColArgs<W> a)
{
    cols_inv_body<W, L, LR, DST, TWIST>(a);
}

// Split path with more column bits than one thread holds (L - LR > 5):
// the top bits run in k_cols_fwd / k_cols_inv with LR' = BLO + LB, and the
// middle bits [BLO, BLO + LB) in these kernels, in place in the wave's
// scratch.  Element x = lo + (k << BLO) + (hi << (BLO + LB)); the node of
// register bit J is x >> (BLO + J + 1) = (hi << (LB - J - 1)) | (k >> (J + 1)),
// so a column's twiddles depend on its top bits hi (read from the plan's
// table).  Forward: after the top bits; inverse (transposed): before them.
template <typename W, int L, int BLO, int LB, int NS, bool TWIST>
__global__ void __launch_bounds__(256) k_cols_mid_fwd(const __grid_constant__ ColArgs<W> a)
{
    constexpr int RC = 1 << LB, LO = L - LB;           // LO: bits outside the register group
    constexpr uint32_t N = 1u << L;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.npairs << LO) return;
    const long long pw = idx >> LO;
    const uint32_t r = (uint32_t)idx & ((1u << LO) - 1u);
    const uint32_t lo = r & ((1u << BLO) - 1u), hi = r >> BLO;
    const uint32_t base = lo + (hi << (BLO + LB));
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        W *p = (s == 0 ? a.dst0 : a.dst1) + (size_t)pw * N;
        W v[RC];
#pragma unroll
        for (int k = 0; k < RC; ++k) v[k] = p[base + ((uint32_t)k << BLO)];
        colf_levels<W, LB, 0, LB - 1, L - BLO - LB, TW_GLOBAL, RC>(v, hi << LB, a.tw, a.c);
        if constexpr (TWIST) {                        // the twist (brv over all L - BLO top bits)
            const uint32_t hbrv = __brev(hi) >> (32 - (L - BLO - LB));
#pragma unroll
            for (int k = 0; k < RC; ++k)
                v[k] = csub<W>(twist<W, L>(v[k], (brv_c32<LB>((uint32_t)k) << (L - BLO - LB)) | hbrv, lo, a, a.pwl), a.c.m);
        }
#pragma unroll
        for (int k = 0; k < RC; ++k) p[base + ((uint32_t)k << BLO)] = v[k];
    }
}

template <typename W, int L, int BLO, int LB, bool TWIST>
__global__ void __launch_bounds__(256) k_cols_mid_inv(const __grid_constant__ ColArgs<W> a)
{
    constexpr int RC = 1 << LB, LO = L - LB;
    constexpr uint32_t N = 1u << L;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.npairs << LO) return;
    const long long pw = idx >> LO;
    const uint32_t r = (uint32_t)idx & ((1u << LO) - 1u);
    const uint32_t lo = r & ((1u << BLO) - 1u), hi = r >> BLO;
    const uint32_t base = lo + (hi << (BLO + LB));
    W *p = a.dst0 + (size_t)pw * N;
    W v[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) v[k] = p[base + ((uint32_t)k << BLO)];
    if constexpr (TWIST) {
        const uint32_t hbrv = __brev(hi) >> (32 - (L - BLO - LB));
#pragma unroll
        for (int k = 0; k < RC; ++k)
            v[k] = twist<W, L>(v[k], (brv_c32<LB>((uint32_t)k) << (L - BLO - LB)) | hbrv, lo, a, a.pwl);
    }
    colg_levels<W, LB, 0, 0, L - BLO - LB, TW_GLOBAL, RC>(v, hi << LB, a.tw, a.c);
#pragma unroll
    for (int k = 0; k < RC; ++k) p[base + ((uint32_t)k << BLO)] = v[k];
}

// Forward row levels of the split path (single sequence, in place in scratch).
template <typename W, int L, int LR>
__global__ void __launch_bounds__(BLOCK, 1) k_rows_fwd(const __grid_constant__ RowArgs<W> a)
{
    using G = Geo<W, LR>;
    constexpr int T = G::T, R = G::R, GPC = RowShape<W, L, LR>::GPC;
    constexpr uint32_t N = 1u << L;
    constexpr int last = G::NPASS - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gid = threadIdx.x / T;
    const uint32_t tau = threadIdx.x % T;
    W *S = reinterpret_cast<W *>(smem_raw) + (size_t)gid * G::ROWP;
    const uint32_t b0 = G::base(0, tau);
    for (long long rho = (long long)blockIdx.x * GPC + gid; rho < a.nrows; rho += (long long)gridDim.x * GPC) {
        const long long pw = rho >> (L - LR);
        const uint32_t row = (uint32_t)rho & ((1u << (L - LR)) - 1u);
        W *p = const_cast<W *>(a.f) + (size_t)pw * N + ((size_t)row << LR);
        W v[1][R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[0][k] = p[b0 + ((uint32_t)k << G::lo(0))];
        fwd_all<W, L, LR, 0, 1, TW_GLOBAL>(v, row << LR, tau, S, gid, a.tw, a.c);
        // back to the first pass's layout, where a warp's stores are contiguous
        if constexpr (last > 0) exchange<W, LR, last, 0, 1>(v, S, tau, gid);
#pragma unroll
        for (int k = 0; k < R; ++k) p[b0 + ((uint32_t)k << G::lo(0))] = v[0][k];
    }
}

// Forward rows of the split path's twist form, for the natural-order
// transforms: after the twisted column pass every row of 2^LR words is a
// whole length-2^LR tree with the uniform table (the first 2^(LR-1) entries
// of the plan's table), staged in shared memory.  In place, tree order: the
// same layout as the row-dependent rows (X(brv(k) + 2^LC brv(j)) at row k,
// position j), so the same bit-reversal gather follows.  32-bit words load
// the next row while this one is transformed.
template <typename W, int LR>
__global__ void __launch_bounds__(BLOCK, 1) k_rows_uni(const __grid_constant__ RowArgs<W> a)
{
    using G = Geo<W, LR>;
    constexpr int T = G::T, R = G::R, GPC = RowShape<W, LR, LR>::GPC;
    constexpr int last = G::NPASS - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gid = threadIdx.x / T;
    const uint32_t tau = threadIdx.x % T;
    W *stw = reinterpret_cast<W *>(smem_raw);
    W *S = reinterpret_cast<W *>(smem_raw + TwBytes<W, LR>::v) + (size_t)gid * G::ROWP;
    const uint32_t b0 = G::base(0, tau);
    stage_twiddles<W>(a.tw, stw, TwBytes<W, LR>::pairs);
    __syncthreads();
    constexpr bool PF = sizeof(W) == 4;
    const long long step = (long long)gridDim.x * GPC;
    long long rho = (long long)blockIdx.x * GPC + gid;
    W v[1][R], w[R];
    auto load = [&](long long r, W (&dst)[R]) {
        const W *p = a.f + ((size_t)r << LR);
#pragma unroll
        for (int k = 0; k < R; ++k) dst[k] = p[b0 + ((uint32_t)k << G::lo(0))];
    };
    if (PF && rho < a.nrows) load(rho, v[0]);
    for (; rho < a.nrows; rho += step) {
        if (!PF) load(rho, v[0]);
        const bool more = PF && rho + step < a.nrows;
        if (more) load(rho + step, w);
        fwd_all<W, LR, LR, 0, 1, TW_SMEM>(v, 0u, tau, S, gid, stw, a.c);
        // back to the first pass's layout, where a warp's stores are contiguous
        if constexpr (last > 0) exchange<W, LR, last, 0, 1>(v, S, tau, gid);
        W *p = const_cast<W *>(a.f) + ((size_t)rho << LR);
#pragma unroll
        for (int k = 0; k < R; ++k) p[b0 + ((uint32_t)k << G::lo(0))] = v[0][k];
        if (more) {
#pragma unroll
            for (int k = 0; k < R; ++k) v[0][k] = w[k];
        }
    }
}

// Bit-reversal gather of a split-path spectrum: y[u] = X(u) from the tree
// order (X(brv(x)) at x); INV applies <-u>_N and N^-1.  Canonical outputs.
template <typename W, int L, bool INV>
__global__ void k_bitrev_out(const W *__restrict__ src, W *__restrict__ dst, long long batch, ModC<W> c)
{
    constexpr uint32_t N = 1u << L;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= batch << L) return;
    const long long b = idx >> L;
    const uint32_t t = (uint32_t)idx & (N - 1u);
    const uint32_t u = INV ? ((N - t) & (N - 1u)) : t;
    const uint32_t x = __brev(u) >> (32 - L);
    const W scale = INV ? c.ninv : (W)1;
    const W scalep = INV ? c.ninvp : c.onep;
    dst[idx] = csub<W>(shoup<W>(src[(size_t)b * N + x], scale, scalep, c.m), c.m);
}

// The same gather, tiled (L >= 10): write an index as (h, m, l) with h and
// l of 5 bits, so brv(h, m, l) = (brv l, brv m, brv h).  For one value of m
// the 32 x 32 elements u = (uh, m, ul) come from x = (brv ul, brv m, brv uh):
// a block reads them as 32 contiguous source runs (fixed brv ul), passes
// them through a padded shared tile, and writes 32 contiguous destination
// runs (fixed uh) -- both directions coalesced.  INV writes u to <-u>_N,
// which keeps every destination run contiguous (descending).
template <typename W, int L, bool INV>
__global__ void __launch_bounds__(256) k_bitrev_tiled(const W *__restrict__ src, W *__restrict__ dst, long long batch,
                                                     ModC<W> c)
{
    static_assert(L >= 10, "two 5-bit ends");
    constexpr uint32_t N = 1u << L;
    constexpr int LM = L - 10;                         // middle bits
    __shared__ W tile[32][33];
    const long long t = blockIdx.x;                    // (sequence, m)
    const long long b = t >> LM;
    const uint32_t m = (uint32_t)t & ((1u << LM) - 1u);
    const uint32_t mb = LM ? (__brev(m) >> (32 - LM)) : 0u;
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const W *s = src + (size_t)b * N;
    W *d = dst + (size_t)b * N;
    const W scale = INV ? c.ninv : (W)1;
    const W scalep = INV ? c.ninvp : c.onep;
    // source runs: x = (sh, mb, sl), sh = brv(ul) fixed per run, sl = lane
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint32_t sh = wid * 4 + r;
        tile[sh][lane] = s[(sh << (L - 5)) | (mb << 5) | lane];
    }
    __syncthreads();
    // destination runs: u = (uh, m, ul), ul = lane; value at x = (brv ul, mb, brv uh)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint32_t uh = wid * 4 + r;
        const uint32_t u = (uh << (L - 5)) | (m << 5) | lane;
        const W v = tile[__brev(lane) >> 27][__brev(uh) >> 27];
        d[INV ? ((N - u) & (N - 1u)) : u] = csub<W>(shoup<W>(v, scale, scalep, c.m), c.m);
    }
}

// ---------------------------------------------------- plain per-stage form

// One forward tree level over the whole batch of f and g: work = [2][batch][N].
template <typename W>
__global__ void k_plain_fwd(const W *__restrict__ f, const W *__restrict__ g, W *work, long long batch,
                            int L, int d, const W *__restrict__ tw, ModC<W> c)
{
    const long long half = 1ll << (L - 1);
    const long long total = 2 * batch * half;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / (batch * half);
        const long long r = i - s * batch * half;
        const long long pair = r >> (L - 1);
        const uint32_t beta = (uint32_t)(r & (half - 1));
        const int sh = L - 1 - d;
        const uint32_t node = beta >> sh;
        const uint32_t i0 = (node << (sh + 1)) | (beta & ((1u << sh) - 1u));
        const uint32_t i1 = i0 + (1u << sh);
        W *dst = work + ((size_t)s * batch + pair) * ((size_t)half * 2);
        W x0, x1;
        if (d == 0) {
            const W *sp = (s == 0 ? f : g) + (size_t)pair * ((size_t)half * 2);
            x0 = sp[i0]; x1 = sp[i1];
            ct_bfly_one<W>(x0, x1, c);
        } else {
            x0 = dst[i0]; x1 = dst[i1];
            const W z = tw[2 * node], zp = tw[2 * node + 1];
            ct_bfly<W>(x0, x1, z, zp, c);
        }
        dst[i0] = x0; dst[i1] = x1;
    }
}

template <typename W>
__global__ void k_plain_pointwise(W *work, long long batch, int L, ModC<W> c)
{
    const long long n = batch << L;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        work[i] = pointwise(work[i], work[n + i], c);
}

template <typename W>
__global__ void k_plain_inv(W *work, long long batch, int L, int d, const W *__restrict__ tw, ModC<W> c)
{
    const long long half = 1ll << (L - 1);
    const long long total = batch * half;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long pair = i >> (L - 1);
        const uint32_t beta = (uint32_t)(i & (half - 1));
        const int sh = L - 1 - d;
        const uint32_t node = beta >> sh;
        const uint32_t i0 = (node << (sh + 1)) | (beta & ((1u << sh) - 1u));
        const uint32_t i1 = i0 + (1u << sh);
        W *p = work + (size_t)pair * ((size_t)half * 2);
        W x0 = p[i0], x1 = p[i1];
        if (d == 0) gs_bfly_one<W>(x0, x1, c);
        else gs_bfly<W>(x0, x1, tw[2 * node], tw[2 * node + 1], c);
        p[i0] = x0; p[i1] = x1;
    }
}

template <typename W>
__global__ void k_plain_final(const W *__restrict__ work, W *h, long long batch, int L, ModC<W> c)
{
    const long long n = batch << L;
    const uint32_t N = 1u << L;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long pair = i >> L;
        const uint32_t x = (uint32_t)i & (N - 1u);
        h[(size_t)pair * N + ((N - x) & (N - 1u))] = csub<W>(work[i], c.m);
    }
}

// Words >= m in data[0 .. n).
template <typename W>
__global__ void k_check_range(const W *__restrict__ data, long long n, W m, unsigned long long *bad)
{
    unsigned long long cnt = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        cnt += data[i] >= m ? 1ull : 0ull;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(bad, cnt);
}

}  // namespace ntt
