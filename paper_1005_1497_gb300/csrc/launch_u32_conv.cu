// Fused-convolution kernel instantiations for 32-bit words.
#include "launch_impl.cuh"
namespace ntt {
template int Launch<uint32_t>::rows_per_block(int);
template int Launch<uint32_t>::pairs_per_block(int, int);
template bool Launch<uint32_t>::block_ok(int, int);
template cudaError_t Launch<uint32_t>::conv_full(int, int, const RowArgs<uint32_t> &, int, cudaStream_t, int);
template cudaError_t Launch<uint32_t>::conv_full_src<0>(int, const RowArgs<uint32_t> &, int, cudaStream_t, int);
template cudaError_t Launch<uint32_t>::conv_small(int, const RowArgs<uint32_t> &, int, cudaStream_t);
}  // namespace ntt
