// The exact convolution's fused kernel instantiations (32-bit words).
#include "launch_impl.cuh"
namespace ntt {
template cudaError_t Launch<uint32_t>::conv_exact(int, bool, const RowArgs<uint32_t> &, const ExactArgs &, int, cudaStream_t);
}  // namespace ntt
