// Executes on host buffers (sfft4_execute_batched_host): the inputs are staged from page-locked
// host memory into the workspace's device copy by a zero-copy kernel, the batch runs as an
// asynchronous execute, and the results are copied back to the host.  The stagings of
// consecutive calls run one after another on the plan's staging stream, so the host link
// stays busy while each batch computes on its workspace's stream.
//
// The staging is a kernel rather than a copy-engine transfer: both reach the host link's rate
// (211 GB/s on a GB300) when alone, but beside the transforms of the previous batch the
// copy-engine transfer was measured at 55-60 GB/s on some machines while 32 CTAs of zero-copy
// loads kept 206-211 GB/s and slowed those transforms by about a fifth.
#include "sfft4_internal.cuh"

namespace {

constexpr int kStageCtas = 32;      // enough loads in flight for the link; the rest of the
constexpr int kStageThreads = 512;  // SMs stay with the previous batch's transforms

// Rows of 2^lg elements of T from src (row stride src_stride elements) into dst (dense rows),
// total = rows x 2^lg elements; four loads in flight per thread.
template <typename T>
__global__ void __launch_bounds__(kStageThreads) k_stage_rows(const T* __restrict__ src, int64_t src_stride,
                                                             T* __restrict__ dst, int64_t total, int lg) {
    const int64_t mask = ((int64_t)1 << lg) - 1;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * step < total; i += 4 * step) {
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = i + u * step;
            v[u] = src[(k >> lg) * src_stride + (k & mask)];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) dst[i + u * step] = v[u];
    }
    for (; i < total; i += step) dst[i] = src[(i >> lg) * src_stride + (i & mask)];
}

int ensure_host_buffers(sfft4_plan_s* w) {
    if (w->hx) return SFFT4_OK;
    const int64_t nb = w->o.max_batch;
    int rc = sfft4::check_cuda(cudaMalloc(&w->hx, (size_t)nb * w->N * sizeof(float2)));
    if (!rc) rc = sfft4::check_cuda(cudaMalloc(&w->hidx, (size_t)nb * w->K * sizeof(int64_t)));
    if (!rc) rc = sfft4::check_cuda(cudaMalloc(&w->hval, (size_t)nb * w->K * sizeof(sfft4_c128)));
    if (!rc) rc = sfft4::check_cuda(cudaMalloc(&w->hnf, (size_t)nb * sizeof(int64_t)));
    if (!rc) rc = sfft4::check_cuda(cudaMalloc(&w->hvotes, (size_t)nb * w->K));
    if (rc) {
        // leave the workspace without a partial set (the next call tries again)
        void* bufs[] = {w->hx, w->hidx, w->hval, w->hnf, w->hvotes};
        for (void* b : bufs) cudaFree(b);
        w->hx = nullptr;
        w->hidx = nullptr;
        w->hval = nullptr;
        w->hnf = nullptr;
        w->hvotes = nullptr;
    }
    return rc;
}

}  // namespace

extern "C" int sfft4_execute_batched_host(sfft4_plan_t p, int32_t nsig, const void* x_host, int64_t x_stride,
                                          int64_t* idx_host, sfft4_c128* val_host, int64_t* nfound_host,
                                          int8_t* votes_host, void* stream) {
    using namespace sfft4;
    if (!p || !x_host || !idx_host || !val_host || !nfound_host) return SFFT4_EINVAL;
    if (p->grp || p->o.trace) return SFFT4_ESTATE;
    if (nsig < 1 || nsig > p->o.max_batch || x_stride < p->N) return SFFT4_EINVAL;
    // the device's address of the page-locked input (none for pageable memory)
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, x_host) != cudaSuccess) {
        (void)cudaGetLastError();
        return SFFT4_EINVAL;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return SFFT4_EINVAL;
    const float2* xd = (const float2*)at.devicePointer;

    int rc = SFFT4_OK;
    if (!p->hstream) rc = check_cuda(cudaStreamCreateWithFlags(&p->hstream, cudaStreamNonBlocking));
    for (int s = 0; s < kAsyncDepth && !rc; ++s)
        if (!p->ev_staged[s]) rc = check_cuda(cudaEventCreateWithFlags(&p->ev_staged[s], cudaEventDisableTiming));
    if (rc) return rc;
    // slot s's previous execute (which read its staged inputs) is ev_done[s] until async_end
    const int s = p->async_next;
    const bool slot_used = (p->async_used >> s) & 1;
    sfft4_plan_s* w = nullptr;
    cudaStream_t as = nullptr;
    rc = async_begin(p, (cudaStream_t)stream, &w, &as);
    if (!rc) rc = ensure_host_buffers(w);
    // staging: after the work queued on `stream` (ev_in[s]) and after slot s's previous
    // execute, behind the previous calls' stagings; the execute waits for it
    if (!rc) rc = check_cuda(cudaStreamWaitEvent(p->hstream, p->ev_in[s], 0));
    if (!rc && slot_used) rc = check_cuda(cudaStreamWaitEvent(p->hstream, p->ev_done[s], 0));
    if (rc) return rc;
    const bool wide = ((uintptr_t)xd % 16 == 0) && (x_stride % 2 == 0);
    if (wide)
        k_stage_rows<uint4><<<kStageCtas, kStageThreads, 0, p->hstream>>>(
            (const uint4*)xd, x_stride / 2, (uint4*)w->hx, (int64_t)nsig * (p->N / 2), p->n - 1);
    else
        k_stage_rows<float2><<<kStageCtas, kStageThreads, 0, p->hstream>>>(xd, x_stride, w->hx,
                                                                           (int64_t)nsig * p->N, p->n);
    rc = check_cuda(cudaGetLastError());
    if (!rc) rc = check_cuda(cudaEventRecord(p->ev_staged[s], p->hstream));
    if (!rc) rc = check_cuda(cudaStreamWaitEvent(as, p->ev_staged[s], 0));
    if (!rc) {
        w->in_async = true;
        rc = run_execute(w, nsig, w->hx, p->N, w->hidx, w->hval, w->hnf, votes_host ? w->hvotes : nullptr, as);
        w->in_async = false;
    }
    const size_t nk = (size_t)nsig * p->K;
    if (!rc) rc = check_cuda(cudaMemcpyAsync(idx_host, w->hidx, nk * sizeof(int64_t), cudaMemcpyDeviceToHost, as));
    if (!rc) rc = check_cuda(cudaMemcpyAsync(val_host, w->hval, nk * sizeof(sfft4_c128), cudaMemcpyDeviceToHost, as));
    if (!rc) rc = check_cuda(cudaMemcpyAsync(nfound_host, w->hnf, (size_t)nsig * sizeof(int64_t),
                                             cudaMemcpyDeviceToHost, as));
    if (!rc && votes_host) rc = check_cuda(cudaMemcpyAsync(votes_host, w->hvotes, nk, cudaMemcpyDeviceToHost, as));
    if (!rc) rc = async_end(p, as);
    return rc;
}
