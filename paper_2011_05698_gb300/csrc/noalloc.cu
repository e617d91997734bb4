// Allocation-free generation of the flat window tables.
//
// sfft4_plan builds the window G and its spectrum G'^ with a temporary FP64 buffer that it
// allocates with cudaMalloc.  Some callers cannot allocate device memory when they need
// these tables: their device memory is owned by another allocator (a framework's caching
// allocator or a fixed pool), or they run latency-critical code that cannot afford the
// implicit device synchronisation of cudaMalloc/cudaFree.  sfft4_window_noalloc computes
// the same tables into caller-provided buffers and uses, as its only scratch, the
// file-scope device array below.
#include <math.h>

#include <mutex>

#include <cuda.h>

#include "sfft4_internal.cuh"

namespace sfft4 {
// Window kernels (defined in kernels.cu).
__global__ void k_window_time(double* g64, int64_t h, int64_t N, int64_t M, double s_t);
__global__ void k_window_norm(const double* g64, int64_t w, float* G32);
__global__ void k_window_spectrum(const float* G32, int64_t h, int64_t N, int n, int64_t nk,
                                  float* Ghat);
}  // namespace sfft4

namespace {

// Largest window (2h + 1 coefficients) the scratch holds: 131072 FP64 values, 1 MiB per
// GPU that loads the library, held until the process exits.  At delta = 1e-8 this covers
// bucket counts up to B = 2048 (w = 90,707).
constexpr int64_t kNoallocMaxW = 131072;
static __device__ __align__(256) double g_window_scratch[kNoallocMaxW];

std::mutex g_setup_mu;
// Per device: the id of the context in which the scratch address was looked up, and the
// address.  A device whose context was destroyed (cudaDeviceReset) and created again gets a
// new context id, so the address is looked up again rather than reused.
struct ScratchCache {
    unsigned long long ctx_id = 0;
    double* ptr = nullptr;
};
ScratchCache g_scratch[64];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Unique id of the calling thread's current CUDA context (0 if none is current yet), through
// the driver entry points the runtime hands out (no link-time dependency on the driver).
// Called with g_setup_mu held.
int current_context_id(unsigned long long* id) {
    *id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        int rc = sfft4::check_cuda(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                                    cudaEnableDefault, &q1));
        if (!rc) rc = sfft4::check_cuda(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000,
                                                                         cudaEnableDefault, &q2));
        if (rc) return rc;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return SFFT4_ECUDA;
        g_ctx_get_current = (CtxGetCurrentFn)f1;
        g_ctx_get_id = (CtxGetIdFn)f2;
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return SFFT4_ECUDA;
    if (!ctx) return SFFT4_OK;
    return g_ctx_get_id(ctx, id) == CUDA_SUCCESS ? SFFT4_OK : SFFT4_ECUDA;
}

// Device address of the scratch array in the current device's current context, looked up
// once per device and context (host code cannot use the symbol itself: it names a host-side
// stand-in, not device memory).
int scratch_address(double** out) {
    int dev = 0;
    int rc = sfft4::check_cuda(cudaGetDevice(&dev));
    if (rc) return rc;
    if (dev < 0 || dev >= 64) return SFFT4_ECUDA;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    unsigned long long id = 0;
    rc = current_context_id(&id);
    if (rc) return rc;
    ScratchCache& c = g_scratch[dev];
    if (id == 0 || c.ctx_id != id || !c.ptr) {
        void* p = nullptr;
        rc = sfft4::check_cuda(cudaGetSymbolAddress(&p, g_window_scratch));  // makes the context current
        if (rc) return rc;
        rc = current_context_id(&id);
        if (rc) return rc;
        c.ctx_id = id;
        c.ptr = (double*)p;
    }
    *out = c.ptr;
    return SFFT4_OK;
}

}  // namespace

extern "C" {

int sfft4_window_noalloc(int64_t N, int32_t B, double delta, float* G_dev, int64_t G_cap,
                         float* Ghat_dev, int64_t Ghat_cap, void* stream) {
    if (N < 256 || (N & (N - 1)) || N > (int64_t(1) << 30)) return SFFT4_EINVAL;
    if (B < sfft4::kBMin || (B & (B - 1)) || B > sfft4::kBMax || B > N / 64) return SFFT4_EINVAL;
    if (!(delta > 0 && delta < 0.5) || !G_dev || !Ghat_dev) return SFFT4_EINVAL;
    int n = 0;
    while ((int64_t(1) << n) < N) ++n;
    double s_t = 0.0;
    const int64_t h = sfft4::window_halfwidth(B, delta, &s_t);
    const int64_t w = 2 * h + 1, L = N / B, nk = (3 * L) / 2 + 1;
    if (w > kNoallocMaxW || w > N / 2) return SFFT4_EINVAL;  // beyond the scratch maximum
    if (G_cap < w || Ghat_cap < nk) return SFFT4_EINVAL;
    double* g64 = nullptr;
    int rc = scratch_address(&g64);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    sfft4::k_window_time<<<(unsigned)((w + 255) / 256), 256, 0, st>>>(g64, h, N, (3 * L) / 4, s_t);
    sfft4::k_window_norm<<<1, 1024, 0, st>>>(g64, w, G_dev);
    sfft4::k_window_spectrum<<<(unsigned)((nk * 32 + 255) / 256), 256, 0, st>>>(G_dev, h, N, n, nk, Ghat_dev);
    return sfft4::check_cuda(cudaGetLastError());
}

}  // extern "C"
