// ntt_noalloc.cu -- conv_circular_noalloc: the batched circular convolution
// for callers that cannot allocate device memory at call time.
//
// Who needs it: code whose device memory is owned entirely by another
// allocator (a framework's caching pool that has reserved the GPU, an
// embedded runtime with a fixed memory map), and latency-critical loops
// that cannot afford cudaMalloc/cudaFree, which may synchronise the whole
// device.  conv_circular keeps its split-path scratch in memory that
// ntt_plan allocates; this entry point instead uses one fixed array that is
// part of the library image on every GPU that loads it, so the call itself
// allocates nothing.  (Creating the plan, which uploads the twiddle table,
// is a set-up step that does allocate; do it during initialisation.  So is
// the first call of this function on a device: it looks up the array's
// device address, and under lazy module loading that lookup is what loads
// this file's module and reserves the array, which can synchronise.)
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ntt_gb300.h"
#include "ntt_internal.h"

namespace {

// Scratch of the split path.  Held by every GPU that loads the library, for
// the life of the process.  Its contents persist between calls.
constexpr size_t kScratchBytes = NTT_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};      // device address of g_noalloc_scratch, per device

// Set-up, once per device with that device current: the host-side name of a
// __device__ array is only a stand-in, so look up its device address.  The
// plan's tables live on the plan's device, so that device must be the
// current one (otherwise the kernels would reach across devices).
ntt_status scratch_address(int plan_dev, void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return ntt_fail(NTT_ERR_CUDA, "conv_circular_noalloc: no usable current device");
    if (dev != plan_dev)
        return ntt_fail(NTT_ERR_ARG, "conv_circular_noalloc: the plan belongs to device %d but device %d is current",
                        plan_dev, dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return ntt_fail(NTT_ERR_CUDA, "conv_circular_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return NTT_OK;
}

}  // namespace

extern "C" ntt_status conv_circular_noalloc(ntt_plan_t plan, const void *f_dev, const void *g_dev, void *h_dev,
                                            size_t batch, ntt_stream_t stream)
{
    if (!plan || !f_dev || !g_dev || !h_dev || batch == 0)
        return ntt_fail(NTT_ERR_ARG, "conv_circular_noalloc: invalid argument");
    ntt_plan_info_t info;
    ntt_status s = ntt_plan_get_info(plan, &info);
    if (s != NTT_OK) return s;
    void *scratch = nullptr;
    uint32_t wave = 0;
    if (info.four_step) {
        // one wave of the split path needs 2 N words per pair
        const size_t per_pair = 2 * (size_t)info.N * (info.word_bits / 8);
        if (per_pair > kScratchBytes)
            return ntt_fail(NTT_ERR_ARG, "conv_circular_noalloc: N=%u needs %zu bytes of scratch per pair, "
                            "above the %zu-byte static scratch", info.N, per_pair, kScratchBytes);
        s = scratch_address(ntt_plan_device(plan), &scratch);
        if (s != NTT_OK) return s;
        size_t w = kScratchBytes / per_pair;
        if (w > batch) w = batch;
        wave = (uint32_t)w;
    }
    // Every scratch word is written by the column pass before the row pass
    // reads it, so nothing has to be cleared between calls.
    return ntt_conv_with_scratch(plan, f_dev, g_dev, h_dev, (long long)batch, scratch, wave, (cudaStream_t)stream);
}
