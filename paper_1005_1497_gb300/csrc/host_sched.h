// host_sched.h -- host-side scheduling rules of the library, plain C++ (no
// CUDA), so that they are also compiled and checked on a host without a GPU
// (tests/host_sched_harness.cpp):
//   - which batches of a one-warp length conv_circular runs with one thread
//     block per pair (k_conv_small) instead of one warp per pair;
//   - how conv_circular_host cuts a batch into the chunks of its copy /
//     convolve / copy-back pipeline.
#pragma once

#include <algorithm>
#include <cstddef>
#include <vector>

namespace ntt {

// Largest batch of length 2^L (L <= rw, the one-warp lengths) that runs one
// block per pair; 0 for longer lengths.  The one-warp kernels win once the
// batch fills the GPU: measured on GB300, the crossover lies near 16 KB of
// input per SM (2^10, 32-bit words: 608 pairs; 64-bit words at 2^9: between
// 608 and 1216), and beyond 32 pairs per SM the block-per-pair kernel's idle
// threads at the shortest lengths cost more.
inline long long small_batch_max(int L, int rw, int word_bytes, int nsm)
{
    if (L > rw || L < 0 || word_bytes <= 0 || nsm <= 0) return 0;
    const long long by_bytes = (long long)nsm * 16384 / ((1LL << L) * word_bytes);
    return std::max<long long>(1, std::min<long long>(by_bytes, (long long)nsm * 32));
}

// Pairs per chunk of the host-buffer pipeline: about 48 MB of input (f and
// g) for whole-sequence lengths, 32 MB on the split path, at least one pair,
// at most the batch.
inline size_t host_chunk_pairs(size_t seq_bytes, bool split, size_t batch)
{
    const size_t bytes = split ? (size_t)32 << 20 : (size_t)48 << 20;
    return std::min(std::max<size_t>(1, bytes / (2 * seq_bytes)), std::max<size_t>(1, batch));
}

// Chunk sizes (pairs) covering `pairs`: full chunks, then 1/2, 1/4 and 1/8
// of one at the end when `shrink_tail` and the batch holds at least four
// full chunks of at least 8 pairs, so that the convolution and outbound copy
// still to run after the last inbound copy are short.
inline std::vector<size_t> host_chunk_sizes(size_t pairs, size_t chunk, bool shrink_tail)
{
    std::vector<size_t> sizes;
    if (chunk == 0) return sizes;
    const size_t tail = (shrink_tail && chunk >= 8 && pairs >= 4 * chunk) ? chunk / 2 + chunk / 4 + chunk / 8 : 0;
    for (size_t body = pairs - tail; body > 0;) {
        const size_t c = std::min(chunk, body);
        sizes.push_back(c);
        body -= c;
    }
    if (tail) sizes.insert(sizes.end(), {chunk / 2, chunk / 4, chunk / 8});
    return sizes;
}

}  // namespace ntt
