// Natural-order transform, plain per-stage form and range-check kernels for 64-bit words.
#include "launch_impl.cuh"
namespace ntt {
template cudaError_t Launch<uint64_t>::ntt_full(int, bool, const NttArgs<uint64_t> &, int, cudaStream_t);
template cudaError_t Launch<uint64_t>::bitrev_out(int, bool, const uint64_t *, uint64_t *, long long,
                                                  const ModC<uint64_t> &, cudaStream_t);
template cudaError_t Launch<uint64_t>::plain(int, const uint64_t *, const uint64_t *, uint64_t *, uint64_t *,
                                             long long, const uint64_t *, const ModC<uint64_t> &, int, cudaStream_t);
template cudaError_t Launch<uint64_t>::check_range(const uint64_t *, long long, uint64_t, unsigned long long *, int,
                                                   cudaStream_t);
}  // namespace ntt
