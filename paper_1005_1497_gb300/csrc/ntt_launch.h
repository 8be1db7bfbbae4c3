// ntt_launch.h -- host-side launchers of the kernels, one instantiation per
// word type (launch_u32.cu / launch_u64.cu).  Internal to the library.
#pragma once

#include <cuda_runtime.h>
#include "ntt_count.h"
#include "ntt_kernels.cuh"

namespace ntt {

template <typename W> struct Launch {
    static constexpr int LRMAX = LRMax<W>::v;
    static constexpr int LMAX = 20;            // split path: LMAX - LRMAX column bits, in two passes above 5
    // rows transformed concurrently by one block of the row kernels
    static int rows_per_block(int LR);
    // pairs in flight per block of the whole-sequence fused kernels with
    // `block` threads per block (BLOCK, or BLOCK_HALF below LRMAX)
    static int pairs_per_block(int L, int block = BLOCK);
    // whether the whole-sequence fused kernels of length 2^L come with `block` threads
    static bool block_ok(int L, int block);
    // whole-sequence fused convolution (L <= LRMAX); src 0 = contiguous, 1 = descriptors
    static cudaError_t conv_full(int L, int src, const RowArgs<W> &a, int grid, cudaStream_t st, int block = BLOCK);
    // (one source mode; instantiated in separate translation units)
    template <int SRC>
    static cudaError_t conv_full_src(int L, const RowArgs<W> &a, int grid, cudaStream_t st, int block);
    // one pair per block (k_conv_small) for the one-warp lengths (L <= RB + 5),
    // contiguous pairs; grid blocks walk the pairs
    static cudaError_t conv_small(int L, const RowArgs<W> &a, int grid, cudaStream_t st);
    static constexpr int SMALL_PER_SM = 8;     // blocks of k_conv_small resident per SM (256 threads, <= 37 registers)
    // split path pieces (LRMAX < L <= LMAX); cols_fwd / cols_inv run one or
    // two column passes
    // (twisted: the four-step twist form, see the twist in ntt_kernels.cuh)
    static cudaError_t conv_rows_split(int L, bool twisted, const RowArgs<W> &a, int grid, cudaStream_t st);
    static cudaError_t cols_fwd(int L, int ns, int src, bool twisted, const ColArgs<W> &a, cudaStream_t st);
    static cudaError_t cols_inv(int L, int dst, bool twisted, const ColArgs<W> &a, cudaStream_t st);
    static cudaError_t rows_fwd(int L, const RowArgs<W> &a, int grid, cudaStream_t st);
    // rows of the twist form for transforms: whole length-2^LRMAX trees in place
    static cudaError_t rows_uni(const RowArgs<W> &a, int grid, cudaStream_t st);
    static cudaError_t bitrev_out(int L, bool inv, const W *src, W *dst, long long batch, const ModC<W> &c,
                                  cudaStream_t st);
    // natural-order transform of whole sequences (L <= LRMAX)
    static cudaError_t ntt_full(int L, bool inv, const NttArgs<W> &a, int grid, cudaStream_t st);
    // plain per-stage form
    static cudaError_t plain(int L, const W *f, const W *g, W *h, W *work, long long batch, const W *tw,
                             const ModC<W> &c, int grid, cudaStream_t st);
    static cudaError_t check_range(const W *data, long long n, W m, unsigned long long *bad, int grid,
                                   cudaStream_t st);
    // the exact convolution's fused launch of one prime (whole sequences,
    // contiguous, signed 64-bit inputs): residues of h to a.h, or (garner)
    // the reconstructed signed 64-bit h to e.h64
    static cudaError_t conv_exact(int L, bool garner, const RowArgs<W> &a, const ExactArgs &e, int grid, cudaStream_t st);
    // dynamic shared memory of the whole-sequence fused kernel of length 2^L
    static size_t conv_full_smem(int L);
    // one persistent launch over a work list of whole-sequence items
    // (lmax: the longest length among the items; selects the instantiation)
    static cudaError_t conv_persistent(const PersistArgs<W> &a, int lmax, int grid, size_t smem, cudaStream_t st);
};

}  // namespace ntt
