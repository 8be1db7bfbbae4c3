// Fused-convolution kernel instantiations for 64-bit words, descriptor-list
// sources (batch plans, the server); a unit of its own for parallel builds.
#include "launch_impl.cuh"
namespace ntt {
template cudaError_t Launch<uint64_t>::conv_full_src<1>(int, const RowArgs<uint64_t> &, int, cudaStream_t, int);
}  // namespace ntt
