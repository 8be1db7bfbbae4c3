// One persistent kernel over every whole-sequence length, 64-bit words.
#include "launch_impl.cuh"
namespace ntt {
template size_t Launch<uint64_t>::conv_full_smem(int);
template cudaError_t Launch<uint64_t>::conv_persistent(const PersistArgs<uint64_t> &, int, int, size_t, cudaStream_t);
}  // namespace ntt
