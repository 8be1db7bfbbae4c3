// One persistent kernel over every whole-sequence length, 32-bit words.
#include "launch_impl.cuh"
namespace ntt {
template size_t Launch<uint32_t>::conv_full_smem(int);
template cudaError_t Launch<uint32_t>::conv_persistent(const PersistArgs<uint32_t> &, int, int, size_t, cudaStream_t);
}  // namespace ntt
