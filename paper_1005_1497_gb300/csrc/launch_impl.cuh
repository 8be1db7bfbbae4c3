// launch_impl.cuh -- template bodies of the launchers (included by the
// per-word-type translation units only).
#pragma once

#include "ntt_launch.h"
#include "ntt_small.cuh"

namespace ntt {

template <typename K>
static cudaError_t ensure_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename W>
int Launch<W>::rows_per_block(int LR)
{
    const int RB = Arith<W>::RB;
    const int RL = LR < RB ? LR : RB;
    return BLOCK >> (LR - RL);
}

// Whole sequences: rows that fit one warp run the warp-level kernel; longer
// ones (up to one block) the column/row kernel.  BLK threads per block.
template <typename W, int L, int SRC, int BLK>
static cudaError_t launch_conv_full_blk(const RowArgs<W> &a, int grid, cudaStream_t st)
{
    constexpr int RW = Arith<W>::RB + 5;
    if constexpr (L <= RW) {
        constexpr size_t smem = TwBytes<W, L>::v + RowShape<W, L, L, BLK>::smem(2);
        static const cudaError_t init = ensure_smem(k_conv_fused<W, L, SRC, BLK>, smem);
        if (init != cudaSuccess) return init;
        k_conv_fused<W, L, SRC, BLK><<<grid, BLK, smem, st>>>(a);
        return launched();
    } else if constexpr (L <= LRMax<W>::v && (BLK == BLOCK || L < LRMax<W>::v)) {
        constexpr size_t smem = CRShape<W, L, L, BLK>::smem;
        static const cudaError_t init = ensure_smem(k_conv_cr<W, L, L, SRC, 0, BLK>, smem);
        if (init != cudaSuccess) return init;
        k_conv_cr<W, L, L, SRC, 0, BLK><<<grid, BLK, smem, st>>>(a);
        return launched();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename W, int L, int SRC>
static cudaError_t launch_conv_full(const RowArgs<W> &a, int grid, cudaStream_t st, int block)
{
    if (block == BLOCK_HALF) return launch_conv_full_blk<W, L, SRC, BLOCK_HALF>(a, grid, st);
    return launch_conv_full_blk<W, L, SRC, BLOCK>(a, grid, st);
}

template <typename W>
bool Launch<W>::block_ok(int L, int block)
{
    if (block == BLOCK) return L >= 0 && L <= LRMAX;
    return block == BLOCK_HALF && L >= 0 && L < LRMAX;
}

template <typename W, int L>
static size_t full_smem_of()
{
    constexpr int RW = Arith<W>::RB + 5;
    if constexpr (L <= RW) return TwBytes<W, L>::v + RowShape<W, L, L>::smem(2);
    else if constexpr (L <= LRMax<W>::v) return CRShape<W, L>::smem;
    else return 0;
}

template <typename W>
size_t Launch<W>::conv_full_smem(int L)
{
    switch (L) {
#define S(X) case X: return full_smem_of<W, X>();
    S(0) S(1) S(2) S(3) S(4) S(5) S(6) S(7) S(8) S(9) S(10) S(11) S(12) S(13) S(14)
#undef S
    default: return 0;
    }
}

template <typename W, int HI>
static cudaError_t launch_persistent(const PersistArgs<W> &a, int grid, size_t smem, cudaStream_t st)
{
    static const cudaError_t init = [] {
        size_t most = 0;
        for (int L = 0; L <= HI; ++L) most = std::max(most, Launch<W>::conv_full_smem(L));
        return cudaFuncSetAttribute(k_conv_persistent<W, HI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    }();
    if (init != cudaSuccess) return init;
    k_conv_persistent<W, HI><<<grid, BLOCK, smem, st>>>(a);
    return launched();
}

template <typename W>
cudaError_t Launch<W>::conv_persistent(const PersistArgs<W> &a, int lmax, int grid, size_t smem, cudaStream_t st)
{
    constexpr int RW = Arith<W>::RB + 5;
    if (lmax <= RW) return launch_persistent<W, RW>(a, grid, smem, st);
    return launch_persistent<W, LRMax<W>::v>(a, grid, smem, st);
}

template <typename W, int L, class X>
static cudaError_t launch_exact(const RowArgs<W> &a, const ExactArgs &e, int grid, cudaStream_t st)
{
    if constexpr (L <= LRMax<W>::v) {
        const size_t smem = full_smem_of<W, L>();
        static const cudaError_t init = ensure_smem(k_conv_exact<W, L, X>, smem);
        if (init != cudaSuccess) return init;
        k_conv_exact<W, L, X><<<grid, BLOCK, smem, st>>>(a, e);
        return launched();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename W>
int Launch<W>::pairs_per_block(int L, int block)
{
    const int RW = Arith<W>::RB + 5;
    if (L <= RW) return rows_per_block(L) * block / BLOCK;
    return block / (32 << (L - RW));
}

// Rows of a convolution's split path.  Untwisted: one row of 2^LR of the
// length-2^L tree, node twiddles from the plan's table (they depend on the
// row).  Twisted: after the twist of the column pass the rows are whole
// length-2^LR convolutions with the uniform table, so one kernel serves
// every L; output lazy, natural order.
template <typename W, int L>
static cudaError_t launch_conv_rows(bool twisted, const RowArgs<W> &a, int grid, cudaStream_t st)
{
    constexpr int LR = LRMax<W>::v;
    if constexpr (L > LR && L <= Launch<W>::LMAX) {
        if (twisted) {
            constexpr size_t smem = CRShape<W, LR, LR>::smem;
            static const cudaError_t init = ensure_smem(k_conv_cr<W, LR, LR, 0, 1>, smem);
            if (init != cudaSuccess) return init;
            k_conv_cr<W, LR, LR, 0, 1><<<grid, BLOCK, smem, st>>>(a);
        } else {
            constexpr size_t smem = CRShape<W, L, LR>::smem;
            static const cudaError_t init = ensure_smem(k_conv_cr<W, L, LR, 0>, smem);
            if (init != cudaSuccess) return init;
            k_conv_cr<W, L, LR, 0><<<grid, BLOCK, smem, st>>>(a);
        }
        return launched();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename W, int L>
static cudaError_t launch_rows_fwd(const RowArgs<W> &a, int grid, cudaStream_t st)
{
    constexpr int LR = LRMax<W>::v;
    if constexpr (L > LR && L <= Launch<W>::LMAX) {
        constexpr size_t smem = RowShape<W, L, LR>::smem(1);
        static const cudaError_t init = ensure_smem(k_rows_fwd<W, L, LR>, smem);
        if (init != cudaSuccess) return init;
        k_rows_fwd<W, L, LR><<<grid, BLOCK, smem, st>>>(a);
        return launched();
    } else {
        return cudaErrorInvalidValue;
    }
}

// Column bits of the split path: up to CMAX in one pass; above that, a top
// pass of L - LR - LB bits and a middle pass of LB = (L - LR) / 2 bits.
constexpr int CMAX = 5;
template <typename W, int L> struct ColSplit {
    static constexpr int LR = LRMax<W>::v;
    static constexpr int LC = L - LR;
    static constexpr bool TWO = LC > CMAX;
    static constexpr int LB = TWO ? LC / 2 : 0;          // middle bits
    static constexpr int TOPLR = LR + LB;                // "row" bits seen by the top pass
};

template <typename W, int L, int NS, int SRC, bool TW>
static cudaError_t launch_cols_fwd(const ColArgs<W> &a, cudaStream_t st)
{
    using CS = ColSplit<W, L>;
    if constexpr (L > CS::LR && L <= Launch<W>::LMAX) {
        const long long threads = a.npairs << CS::TOPLR;
        k_cols_fwd<W, L, CS::TOPLR, NS, SRC, TW && !CS::TWO><<<(int)((threads + 255) / 256), 256, 0, st>>>(a);
        if constexpr (CS::TWO) {
            const long long t2 = a.npairs << (L - CS::LB);
            k_cols_mid_fwd<W, L, CS::LR, CS::LB, NS, TW><<<(int)((t2 + 255) / 256), 256, 0, st>>>(a);
        }
        return launched(CS::TWO ? 2 : 1);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename W, int L, int DST, bool TW>
static cudaError_t launch_cols_inv(const ColArgs<W> &a, cudaStream_t st)
{
    using CS = ColSplit<W, L>;
    if constexpr (L > CS::LR && L <= Launch<W>::LMAX) {
        if constexpr (CS::TWO) {
            const long long t2 = a.npairs << (L - CS::LB);
            k_cols_mid_inv<W, L, CS::LR, CS::LB, TW><<<(int)((t2 + 255) / 256), 256, 0, st>>>(a);
        }
        const long long threads = a.npairs << CS::TOPLR;
        if constexpr (sizeof(W) == 4 && L - CS::TOPLR == 5)
            k_cols_inv5<W, L, CS::TOPLR, DST, TW && !CS::TWO><<<(int)((threads + 255) / 256), 256, 0, st>>>(a);
        else
            k_cols_inv<W, L, CS::TOPLR, DST, TW && !CS::TWO><<<(int)((threads + 255) / 256), 256, 0, st>>>(a);
        return launched(CS::TWO ? 2 : 1);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename W, int L, bool INV>
static cudaError_t launch_ntt_full(const NttArgs<W> &a, int grid, cudaStream_t st)
{
    if constexpr (L <= LRMax<W>::v) {
        constexpr size_t smem = TwBytes<W, L>::v + RowShape<W, L, L>::smem(1);
        static const cudaError_t init = ensure_smem(k_ntt_rows<W, L, INV>, smem);
        if (init != cudaSuccess) return init;
        k_ntt_rows<W, L, INV><<<grid, BLOCK, smem, st>>>(a);
        return launched();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename W, int L, bool INV>
static cudaError_t launch_bitrev(const W *src, W *dst, long long batch, const ModC<W> &c, cudaStream_t st)
{
    if constexpr (L >= 10) {
        const long long tiles = batch << (L - 10);
        k_bitrev_tiled<W, L, INV><<<(unsigned)tiles, 256, 0, st>>>(src, dst, batch, c);
        return launched();
    } else if constexpr (L >= 1) {
        const long long n = batch << L;
        k_bitrev_out<W, L, INV><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, batch, c);
        return launched();
    } else {
        return cudaErrorInvalidValue;
    }
}

#define NTT_SWITCH_L(CALL)                                                               \
    switch (L) {                                                                         \
    case 0: return CALL(0); case 1: return CALL(1); case 2: return CALL(2);              \
    case 3: return CALL(3); case 4: return CALL(4); case 5: return CALL(5);              \
    case 6: return CALL(6); case 7: return CALL(7); case 8: return CALL(8);              \
    case 9: return CALL(9); case 10: return CALL(10); case 11: return CALL(11);          \
    case 12: return CALL(12); case 13: return CALL(13); case 14: return CALL(14);        \
    case 15: return CALL(15); case 16: return CALL(16); case 17: return CALL(17);        \
    case 18: return CALL(18); case 19: return CALL(19); case 20: return CALL(20);        \
    default: return cudaErrorInvalidValue;                                               \
    }

template <typename W>
template <int SRC>
cudaError_t Launch<W>::conv_full_src(int L, const RowArgs<W> &a, int grid, cudaStream_t st, int block)
{
#define C(X) launch_conv_full<W, X, SRC>(a, grid, st, block)
    NTT_SWITCH_L(C)
#undef C
}

template <typename W, int L>
static cudaError_t launch_conv_small(const RowArgs<W> &a, int grid, cudaStream_t st)
{
    if constexpr (L <= Arith<W>::RB + 5) {
        constexpr size_t smem = SmallShape<W, L>::smem;
        static const cudaError_t init = ensure_smem(k_conv_small<W, L>, smem);
        if (init != cudaSuccess) return init;
        k_conv_small<W, L><<<grid, SMALL_THREADS, smem, st>>>(a);
        return launched();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename W>
cudaError_t Launch<W>::conv_small(int L, const RowArgs<W> &a, int grid, cudaStream_t st)
{
#define C(X) launch_conv_small<W, X>(a, grid, st)
    NTT_SWITCH_L(C)
#undef C
}

template <typename W>
cudaError_t Launch<W>::conv_full(int L, int src, const RowArgs<W> &a, int grid, cudaStream_t st, int block)
{
    if (!block_ok(L, block)) return cudaErrorInvalidValue;
    return src == 1 ? conv_full_src<1>(L, a, grid, st, block) : conv_full_src<0>(L, a, grid, st, block);
}

template <typename W>
cudaError_t Launch<W>::conv_exact(int L, bool garner, const RowArgs<W> &a, const ExactArgs &e, int grid, cudaStream_t st)
{
    if (garner) {
#define C(X) launch_exact<W, X, ExactGarner>(a, e, grid, st)
        NTT_SWITCH_L(C)
#undef C
    }
#define C(X) launch_exact<W, X, ExactResidues>(a, e, grid, st)
    NTT_SWITCH_L(C)
#undef C
}

template <typename W>
cudaError_t Launch<W>::conv_rows_split(int L, bool twisted, const RowArgs<W> &a, int grid, cudaStream_t st)
{
#define C(X) launch_conv_rows<W, X>(twisted, a, grid, st)
    NTT_SWITCH_L(C)
#undef C
}

template <typename W>
cudaError_t Launch<W>::rows_fwd(int L, const RowArgs<W> &a, int grid, cudaStream_t st)
{
#define C(X) launch_rows_fwd<W, X>(a, grid, st)
    NTT_SWITCH_L(C)
#undef C
}

template <typename W>
cudaError_t Launch<W>::rows_uni(const RowArgs<W> &a, int grid, cudaStream_t st)
{
    constexpr int LR = LRMax<W>::v;
    constexpr size_t smem = TwBytes<W, LR>::v + RowShape<W, LR, LR>::smem(1);
    static const cudaError_t init = ensure_smem(k_rows_uni<W, LR>, smem);
    if (init != cudaSuccess) return init;
    k_rows_uni<W, LR><<<grid, BLOCK, smem, st>>>(a);
    return launched();
}

template <typename W>
cudaError_t Launch<W>::cols_fwd(int L, int ns, int src, bool twisted, const ColArgs<W> &a, cudaStream_t st)
{
    if (ns == 2 && src == 0 && twisted) {
#define C(X) launch_cols_fwd<W, X, 2, 0, true>(a, st)
        NTT_SWITCH_L(C)
#undef C
    } else if (ns == 2 && src == 0) {
#define C(X) launch_cols_fwd<W, X, 2, 0, false>(a, st)
        NTT_SWITCH_L(C)
#undef C
    } else if (ns == 2 && src == 1 && twisted) {
#define C(X) launch_cols_fwd<W, X, 2, 1, true>(a, st)
        NTT_SWITCH_L(C)
#undef C
    } else if (ns == 2 && src == 1) {
#define C(X) launch_cols_fwd<W, X, 2, 1, false>(a, st)
        NTT_SWITCH_L(C)
#undef C
    } else if (ns == 1 && src == 0 && !twisted) {
#define C(X) launch_cols_fwd<W, X, 1, 0, false>(a, st)
        NTT_SWITCH_L(C)
#undef C
    } else if (ns == 1 && src == 0) {
#define C(X) launch_cols_fwd<W, X, 1, 0, true>(a, st)
        NTT_SWITCH_L(C)
#undef C
    }
    return cudaErrorInvalidValue;
}

template <typename W>
cudaError_t Launch<W>::cols_inv(int L, int dst, bool twisted, const ColArgs<W> &a, cudaStream_t st)
{
    if (dst == 1 && twisted) {
#define C(X) launch_cols_inv<W, X, 1, true>(a, st)
        NTT_SWITCH_L(C)
#undef C
    } else if (dst == 1) {
#define C(X) launch_cols_inv<W, X, 1, false>(a, st)
        NTT_SWITCH_L(C)
#undef C
    } else if (twisted) {
#define C(X) launch_cols_inv<W, X, 0, true>(a, st)
        NTT_SWITCH_L(C)
#undef C
    }
#define C(X) launch_cols_inv<W, X, 0, false>(a, st)
    NTT_SWITCH_L(C)
#undef C
}

template <typename W>
cudaError_t Launch<W>::ntt_full(int L, bool inv, const NttArgs<W> &a, int grid, cudaStream_t st)
{
    if (inv) {
#define C(X) launch_ntt_full<W, X, true>(a, grid, st)
        NTT_SWITCH_L(C)
#undef C
    }
#define C(X) launch_ntt_full<W, X, false>(a, grid, st)
    NTT_SWITCH_L(C)
#undef C
}

template <typename W>
cudaError_t Launch<W>::bitrev_out(int L, bool inv, const W *src, W *dst, long long batch, const ModC<W> &c,
                                  cudaStream_t st)
{
    if (inv) {
#define C(X) launch_bitrev<W, X, true>(src, dst, batch, c, st)
        NTT_SWITCH_L(C)
#undef C
    }
#define C(X) launch_bitrev<W, X, false>(src, dst, batch, c, st)
    NTT_SWITCH_L(C)
#undef C
}

template <typename W>
cudaError_t Launch<W>::plain(int L, const W *f, const W *g, W *h, W *work, long long batch, const W *tw,
                             const ModC<W> &c, int grid, cudaStream_t st)
{
    const int threads = 256;
    if (L == 0) {
        // N = 1: the convolution is the single product
        cudaError_t e = cudaMemcpyAsync(work, f, sizeof(W) * batch, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(work + batch, g, sizeof(W) * batch, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    } else {
        for (int d = 0; d < L; ++d) {
            k_plain_fwd<W><<<grid, threads, 0, st>>>(f, g, work, batch, L, d, tw, c);
            cudaError_t e = launched();
            if (e != cudaSuccess) return e;
        }
    }
    k_plain_pointwise<W><<<grid, threads, 0, st>>>(work, batch, L, c);
    for (int d = L - 1; d >= 0; --d) k_plain_inv<W><<<grid, threads, 0, st>>>(work, batch, L, d, tw, c);
    k_plain_final<W><<<grid, threads, 0, st>>>(work, h, batch, L, c);
    return launched(L + 2);
}

template <typename W>
cudaError_t Launch<W>::check_range(const W *data, long long n, W m, unsigned long long *bad, int grid,
                                   cudaStream_t st)
{
    k_check_range<W><<<grid, 256, 0, st>>>(data, n, m, bad);
    return launched();
}

}  // namespace ntt
