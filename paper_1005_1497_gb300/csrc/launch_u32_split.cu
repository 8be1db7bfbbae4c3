// Split-path (columns + rows) kernel instantiations for 32-bit words.
#include "launch_impl.cuh"
namespace ntt {
template cudaError_t Launch<uint32_t>::conv_rows_split(int, bool, const RowArgs<uint32_t> &, int, cudaStream_t);
template cudaError_t Launch<uint32_t>::cols_fwd(int, int, int, bool, const ColArgs<uint32_t> &, cudaStream_t);
template cudaError_t Launch<uint32_t>::cols_inv(int, int, bool, const ColArgs<uint32_t> &, cudaStream_t);
template cudaError_t Launch<uint32_t>::rows_fwd(int, const RowArgs<uint32_t> &, int, cudaStream_t);
template cudaError_t Launch<uint32_t>::rows_uni(const RowArgs<uint32_t> &, int, cudaStream_t);
}  // namespace ntt
