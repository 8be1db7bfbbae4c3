// ntt_internal.h -- functions shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include "../../include/ntt_gb300.h"

namespace ntt {
// An NVTX range for the lifetime of the object: plan creation, dispatch,
// batch execution and graph replay, and the server's batches show up as
// named ranges in a profiler's timeline (NVTX does nothing when no tool is
// attached).
struct Trace {
    explicit Trace(const char *name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
    Trace(const Trace &) = delete;
    Trace &operator=(const Trace &) = delete;
};

// cudaMalloc that leaves no error behind when it fails: the library checks
// every launch with cudaGetLastError(), which would otherwise report the
// failed allocation again at the next (good) launch of this thread.
template <typename T>
inline bool dev_alloc(T **p, size_t bytes)
{
    if (cudaMalloc(reinterpret_cast<void **>(p), bytes) == cudaSuccess) return true;
    *p = nullptr;
    (void)cudaGetLastError();
    return false;
}
}  // namespace ntt

// Record a message for ntt_last_error() and return s.
ntt_status ntt_fail(ntt_status s, const char *fmt, ...);
// log2 N of a plan.
int ntt_plan_log2(ntt_plan_t p);
// The device a plan was created on (its tables live there).
int ntt_plan_device(ntt_plan_t p);
// Library-owned plan for (m, N), created on first use.
ntt_status ntt_cached_plan(uint64_t m, uint32_t N, ntt_plan_t *out);
// Fused convolution of `count` pairs given by a device descriptor list
// {f, g, h} (three device pointers each); scratch/wave serve the split path.
ntt_status ntt_conv_descs(ntt_plan_t p, const void *descs_dev, long long count, void *scratch, uint32_t wave,
                          cudaStream_t st);
// Fused convolution of contiguous [batch][N] arrays with caller-chosen
// split-path scratch (wave pairs of 2 N words); scratch unused when N fits one block.
ntt_status ntt_conv_with_scratch(ntt_plan_t p, const void *f, const void *g, void *h, long long batch,
                                 void *scratch, uint32_t wave, cudaStream_t st, int twist = -1);   // twist: -1 the plan's form, 0 / 1 forced
// The autotuned schedule of (this GPU, word size, log2 N); false if none.
struct ntt_schedule_t {
    uint32_t wave;          // split path: pairs per scratch wave
    int twist;              // split path: 1 the four-step twist form, 0 row-dependent twiddles
    int block;              // whole sequences: threads per block of the fused kernel
    int persist;            // whole sequences: 1 when a batch plan runs the length in its persistent launch
};
bool ntt_tuned_schedule(int word_bits, int log2N, ntt_schedule_t *out);
// Threads per block of a whole-sequence plan's fused kernel (the autotuner's
// trial setting); false if the length has no such choice.
bool ntt_plan_set_block(ntt_plan_t p, int block);
// The untuned threads per block of the whole-sequence fused kernel of length 2^L.
int ntt_default_block(int word_bits, int L);
// Device twiddle table of a plan, and its arithmetic constants (ModC<W> of
// the plan's word size copied to out, `bytes` bytes).
// One persistent launch of the whole-sequence fused bodies over a work list
// (device pointers: descs, items, counter (zeroed here), class params).
ntt_status ntt_launch_persistent(int word_bits, const void *descs, const void *items, int nitems, int *counter,
                                 const ntt_plan_t *plans, int lmax, int grid, size_t smem, cudaStream_t st);   // plans: indexed by log2 N, null where absent
size_t ntt_full_smem(int word_bits, int log2N);
bool ntt_persist_class(int word_bits, int L);
// the exact convolution's fused launch of one prime (32-bit plans of whole
// sequences); exact_args: an ntt::ExactArgs
ntt_status ntt_launch_exact(ntt_plan_t p, bool garner, const void *f64, const void *g64, void *h, const void *exact_args,
                            long long np, cudaStream_t st);   // longest length a batch plan runs in its persistent launch
int ntt_num_sms();
