// ntt_count.h -- the library's host-side count of the kernel launches it has
// enqueued (ntt_launch_count).  Internal to the library.
#pragma once

#include <atomic>
#include <cuda_runtime.h>

namespace ntt {

extern std::atomic<unsigned long long> launch_count;

// Record n kernel launches just issued and return the launch status.
inline cudaError_t launched(unsigned n = 1)
{
    launch_count.fetch_add(n, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace ntt
