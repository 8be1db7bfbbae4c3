// Fused-convolution kernel instantiations for 64-bit words.
#include "launch_impl.cuh"
namespace ntt {
template int Launch<uint64_t>::rows_per_block(int);
template int Launch<uint64_t>::pairs_per_block(int, int);
template bool Launch<uint64_t>::block_ok(int, int);
template cudaError_t Launch<uint64_t>::conv_full(int, int, const RowArgs<uint64_t> &, int, cudaStream_t, int);
template cudaError_t Launch<uint64_t>::conv_full_src<0>(int, const RowArgs<uint64_t> &, int, cudaStream_t, int);
template cudaError_t Launch<uint64_t>::conv_small(int, const RowArgs<uint64_t> &, int, cudaStream_t);
}  // namespace ntt
