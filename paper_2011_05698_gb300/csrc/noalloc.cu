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
double* g_scratch_ptr[64] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
int scratch_address(double** out) {
    int dev = 0;
    int rc = sfft4::check_cuda(cudaGetDevice(&dev));
    if (rc) return rc;
    if (dev < 0 || dev >= 64) return SFFT4_ECUDA;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        rc = sfft4::check_cuda(cudaGetSymbolAddress(&p, g_window_scratch));
        if (rc) return rc;
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return SFFT4_OK;
}

double erfcinv_newton(double y) {
    double x = sqrt(-log(y));
    for (int i = 0; i < 100; ++i) {
        double f = erfc(x) - y;
        double d = -2.0 / sqrt(M_PI) * exp(-x * x);
        double step = f / d;
        x -= step;
        if (fabs(step) <= 1e-17 * fabs(x)) break;
    }
    return x;
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
    const double c = 4.0 * sqrt(2.0) * erfcinv_newton(delta);
    const double s_t = (double)B * c / (2.0 * M_PI);
    const int64_t h = (int64_t)ceil(s_t * sqrt(2.0 * log(1.0 / delta)));
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
