// Random-gather throughput probe: the achievable rate of the fold's memory access pattern
// (independent random 8-byte loads within each signal of a batch) on the current device,
// used as the denominator of the gather's roofline.  Every load index is a hash masked to
// the signal's length, so all loads stay inside the caller's buffer.
#include "sfft4_internal.cuh"

namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Block b reads only signal (b mod nsig); each thread issues `iters` x 4 independent loads.
__global__ void k_gather_probe(const float2* __restrict__ x, uint32_t mask, int64_t stride,
                               int nsig, int iters, float* sink) {
    const float2* base = x + (int64_t)(blockIdx.x % nsig) * stride;
    uint32_t st = mix32((blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u);
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            st = st * 1664525u + 1013904223u;
            const uint32_t i = mix32(st) & mask;
            asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v[u].x), "=f"(v[u].y) : "l"(base + i));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc += v[u].x + v[u].y;
    }
    if (acc == 1.2345e-30f) sink[0] = acc;  // keeps the loads; practically never taken
}

}  // namespace

extern "C" {

int sfft4_gather_probe(const void* x_dev, int32_t nsig, int64_t N, int64_t x_stride, float* sink_dev,
                       int32_t blocks, int32_t iters, double* loads_per_second, void* stream) {
    if (!x_dev || !sink_dev || !loads_per_second || nsig < 1 || N < 256 || (N & (N - 1)) ||
        N > (int64_t(1) << 30) || x_stride < N || blocks < 1 || iters < 1)
        return SFFT4_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = sfft4::check_cuda(cudaEventCreate(&a));
    if (!rc) rc = sfft4::check_cuda(cudaEventCreate(&b));
    if (rc) {
        if (a) cudaEventDestroy(a);
        return rc;
    }
    const uint32_t mask = (uint32_t)(N - 1);
    k_gather_probe<<<blocks, 512, 0, st>>>((const float2*)x_dev, mask, x_stride, nsig, 2, sink_dev);
    cudaEventRecord(a, st);
    k_gather_probe<<<blocks, 512, 0, st>>>((const float2*)x_dev, mask, x_stride, nsig, iters, sink_dev);
    cudaEventRecord(b, st);
    rc = sfft4::check_cuda(cudaEventSynchronize(b));
    float ms = 0.f;
    if (!rc) rc = sfft4::check_cuda(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    *loads_per_second = (double)blocks * 512.0 * iters * 4.0 / (ms * 1e-3);
    return SFFT4_OK;
}

}  // extern "C"
