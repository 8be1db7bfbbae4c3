// Natural-order transform, plain per-stage form and range-check kernels for 32-bit words.
#include "launch_impl.cuh"
namespace ntt {
template cudaError_t Launch<uint32_t>::ntt_full(int, bool, const NttArgs<uint32_t> &, int, cudaStream_t);
template cudaError_t Launch<uint32_t>::bitrev_out(int, bool, const uint32_t *, uint32_t *, long long,
                                                  const ModC<uint32_t> &, cudaStream_t);
template cudaError_t Launch<uint32_t>::plain(int, const uint32_t *, const uint32_t *, uint32_t *, uint32_t *,
                                             long long, const uint32_t *, const ModC<uint32_t> &, int, cudaStream_t);
template cudaError_t Launch<uint32_t>::check_range(const uint32_t *, long long, uint32_t, unsigned long long *, int,
                                                   cudaStream_t);
}  // namespace ntt
