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

// Block b reads only signal (b mod nsig); each thread issues `iters` x U independent loads,
// U in flight at a time.
template <int U>
__global__ void k_gather_probe(const float2* __restrict__ x, uint32_t mask, int64_t stride,
                               int nsig, int iters, float* sink) {
    const float2* base = x + (int64_t)(blockIdx.x % nsig) * stride;
    uint32_t st = mix32((blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u);
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        float2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            st = st * 1664525u + 1013904223u;
            const uint32_t i = mix32(st) & mask;
            asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v[u].x), "=f"(v[u].y) : "l"(base + i));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc += v[u].x + v[u].y;
    }
    if (acc == 1.2345e-30f) sink[0] = acc;  // keeps the loads; practically never taken
}

int launch_probe(int U, int blocks, int threads, cudaStream_t st, const float2* x, uint32_t mask, int64_t stride,
                 int nsig, int iters, float* sink) {
    switch (U) {
        case 4: k_gather_probe<4><<<blocks, threads, 0, st>>>(x, mask, stride, nsig, iters, sink); break;
        case 8: k_gather_probe<8><<<blocks, threads, 0, st>>>(x, mask, stride, nsig, iters, sink); break;
        default: k_gather_probe<16><<<blocks, threads, 0, st>>>(x, mask, stride, nsig, iters, sink); break;
    }
    return sfft4::check_cuda(cudaGetLastError());
}

}  // namespace

extern "C" {

int sfft4_gather_probe_ex(const void* x_dev, int32_t nsig, int64_t N, int64_t x_stride, float* sink_dev,
                          int32_t blocks, int32_t threads, int32_t iters, int32_t inflight,
                          int32_t l2_fetch_bytes, double* loads_per_second, void* stream) {
    if (!x_dev || !sink_dev || !loads_per_second || nsig < 1 || N < 256 || (N & (N - 1)) ||
        N > (int64_t(1) << 30) || x_stride < N || blocks < 1 || iters < 1)
        return SFFT4_EINVAL;
    if ((inflight != 4 && inflight != 8 && inflight != 16) || threads < 32 || threads > 1024 || threads % 32)
        return SFFT4_EINVAL;
    if (l2_fetch_bytes != 0 && l2_fetch_bytes != 32 && l2_fetch_bytes != 64 && l2_fetch_bytes != 128)
        return SFFT4_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    size_t old_fetch = 0;
    int rc = SFFT4_OK;
    if (l2_fetch_bytes) {
        rc = sfft4::check_cuda(cudaDeviceGetLimit(&old_fetch, cudaLimitMaxL2FetchGranularity));
        if (!rc) rc = sfft4::check_cuda(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)l2_fetch_bytes));
        if (rc) return rc;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    rc = sfft4::check_cuda(cudaEventCreate(&a));
    if (!rc) rc = sfft4::check_cuda(cudaEventCreate(&b));
    const uint32_t mask = (uint32_t)(N - 1);
    const float2* x = (const float2*)x_dev;
    if (!rc) rc = launch_probe(inflight, blocks, threads, st, x, mask, x_stride, nsig, 2, sink_dev);
    if (!rc) rc = sfft4::check_cuda(cudaEventRecord(a, st));
    if (!rc) rc = launch_probe(inflight, blocks, threads, st, x, mask, x_stride, nsig, iters, sink_dev);
    if (!rc) rc = sfft4::check_cuda(cudaEventRecord(b, st));
    if (!rc) rc = sfft4::check_cuda(cudaEventSynchronize(b));
    float ms = 0.f;
    if (!rc) rc = sfft4::check_cuda(cudaEventElapsedTime(&ms, a, b));
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (l2_fetch_bytes) {
        const int rc2 = sfft4::check_cuda(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, old_fetch));
        if (!rc) rc = rc2;
    }
    if (rc) return rc;
    *loads_per_second = (double)blocks * threads * iters * inflight / (ms * 1e-3);
    return SFFT4_OK;
}

int sfft4_gather_probe(const void* x_dev, int32_t nsig, int64_t N, int64_t x_stride, float* sink_dev,
                       int32_t blocks, int32_t iters, double* loads_per_second, void* stream) {
    return sfft4_gather_probe_ex(x_dev, nsig, N, x_stride, sink_dev, blocks, 512, iters, 4, 0, loads_per_second,
                                 stream);
}

}  // extern "C"
