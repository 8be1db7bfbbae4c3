// int_pipes_probe.cu -- throughput of the integer operations that bound the
// butterflies, the basis of the integer roofline the benchmark reports:
// independent chains per thread of (a) 32-bit multiply-add, (b) the high
// half of a 32 x 32 product (umulhi), (c) a Shoup product (umulhi + two
// multiplies), (d) a lazy Cooley-Tukey butterfly.  Every thread writes one
// word of its own, so all accesses are in bounds.  Built and run by
// test_gpu_int_pipes.py; prints one "name value" pair per line.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#define CH 16

__global__ void k_imad(uint32_t *out, uint32_t a, uint32_t b, int iters)
{
    uint32_t v[CH];
#pragma unroll
    for (int i = 0; i < CH; i++) v[i] = threadIdx.x * 7 + i * 13 + blockIdx.x;
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < CH; i++) v[i] = v[i] * a + b;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < CH; i++) s ^= v[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_mulhi(uint32_t *out, uint32_t a, int iters)
{
    uint32_t v[CH];
#pragma unroll
    for (int i = 0; i < CH; i++) v[i] = threadIdx.x * 7 + i * 13 + blockIdx.x;
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < CH; i++) v[i] = __umulhi(v[i], a) ^ (uint32_t)i;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < CH; i++) s ^= v[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_shoup(uint32_t *out, uint32_t w, uint32_t wp, uint32_t m, int iters)
{
    uint32_t v[CH];
#pragma unroll
    for (int i = 0; i < CH; i++) v[i] = threadIdx.x * 7 + i * 13 + blockIdx.x;
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < CH; i++) v[i] = v[i] * w - __umulhi(v[i], wp) * m;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < CH; i++) s ^= v[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_bfly(uint32_t *out, uint32_t w, uint32_t wp, uint32_t m, int iters)
{
    uint32_t v[CH];
#pragma unroll
    for (int i = 0; i < CH; i++) v[i] = (threadIdx.x * 7 + i * 13 + blockIdx.x) % m;
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < CH; i += 2) {
            uint32_t t = v[i + 1] * w - __umulhi(v[i + 1], wp) * m;
            uint32_t a = v[i];
            v[i] = a + t;
            v[i + 1] = a - t + 2 * m;
        }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < CH; i++) s ^= v[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main()
{
    int nsm = 0, khz = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, 0);
    const int threads = 256, blocks = nsm * 8, iters = 4096;
    uint32_t *out;
    if (cudaMalloc(&out, (size_t)blocks * threads * 4) != cudaSuccess) return 1;
    const uint32_t m = 13631489u, w = 1048261u, wp = (uint32_t)(((uint64_t)w << 32) / m);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const double n = (double)blocks * threads * iters * CH;
    float ms;
    for (int rep = 0; rep < 2; rep++) {
        cudaEventRecord(e0); k_imad<<<blocks, threads>>>(out, w, wp, iters); cudaEventRecord(e1); cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep) printf("imad_per_s %.4e\nimad_per_sm_clk %.2f\n", n / ms * 1e3, n / ms * 1e3 / nsm / (khz * 1e3));
        cudaEventRecord(e0); k_mulhi<<<blocks, threads>>>(out, wp, iters); cudaEventRecord(e1); cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep) printf("umulhi_per_s %.4e\n", n / ms * 1e3);
        cudaEventRecord(e0); k_shoup<<<blocks, threads>>>(out, w, wp, m, iters); cudaEventRecord(e1); cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep) printf("shoup_per_s %.4e\n", n / ms * 1e3);
        cudaEventRecord(e0); k_bfly<<<blocks, threads>>>(out, w, wp, m, iters); cudaEventRecord(e1); cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep) printf("butterfly_per_s %.4e\n", n / 2 / ms * 1e3);
    }
    cudaError_t err = cudaGetLastError();
    printf("sms %d\nclock_khz %d\nstatus %s\n", nsm, khz, cudaGetErrorString(err));
    return err != cudaSuccess;
}
