// B-point DFT of the bucketization (Lemma 1, step P3) as a BF16x3 split-precision complex
// GEMM on the 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// A B-point DFT is composed of at most two stages (four-step: B = B1 B2 with 8 <= B1, B2 <= 64):
//   stage 1: for every (column, j2): u[k1] = sum_j1 W_B1^{j1 k1} z[B2 j1 + j2]
//   stage 2: for every (column, k1): y[k1 + B1 k2] = sum_j2 W_B2^{j2 k2} (W_B^{j2 k1} u_{j2}[k1])
// Each stage applies a P-point complex DFT to many vectors.  In real form a P-point DFT is the
// 2P x 2P matrix [[Wr, -Wi], [Wi, Wr]] acting on [re; im]; 64/P copies are stacked block-
// diagonally into one 128 x 128 matrix A, so every stage is the same GEMM
// D[128 x n] = A[128 x 128] X[128 x n] with 64/P vectors stacked per GEMM column.
// BF16x3: A and X are split into three bf16 pieces (a = a1 + a2 + a3, each the bf16 rounding
// of the remainder) and the six products of order <= 2 (a1x1, a1x2, a2x1, a1x3, a2x2, a3x1)
// accumulate in FP32 in tensor memory, so the result carries FP32-level error.
#include <math.h>
#include <stdio.h>

#include <cuda_bf16.h>

#include "sfft4_internal.cuh"

namespace sfft4 {

namespace {

constexpr int kM = 128, kK = 128, kNT = 128;       // GEMM tile: M x K x N
constexpr int kPieceBytes = kM * kK * 2;            // one bf16 128 x 128 operand
constexpr int kDftSmem = 6 * kPieceBytes + 1024;    // 3 A pieces + 3 X pieces + alignment
constexpr int kDftThreads = 512;  // 4 warpgroups; warp w reads TMEM lanes 32 (w % 4) ..
constexpr uint32_t kWaitLimit = 1u << 24;           // mbarrier polls before giving up

// Byte offset of element (r, k) of an R x 128 K-major bf16 operand stored as 8 x 16-byte core
// matrices: core (r/8, k/8) at ((r/8) 16 + k/8) 128, row r%8 at +16 (r%8), column k%8 at +2 (k%8).
// In the tcgen05 shared-memory descriptor this is leading-byte offset 128 (next core matrix
// along K) and stride-byte offset 2048 (next core matrix along M or N), no swizzle.
__host__ __device__ __forceinline__ int core_off(int r, int k) {
    return (((r >> 3) * (kK / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;    // leading-byte offset: next core matrix along K
    d |= (uint64_t)(2048u >> 4) << 32;   // stride-byte offset: next core matrix along M / N
    d |= (uint64_t)1 << 46;              // descriptor version of tcgen05
    return d;                            // base offset 0, no swizzle
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, N = kNT, M = kM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kNT >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

// A = block-diagonal stack of 64/P real-form P-point DFT matrices, split into three bf16 pieces
// (FP64 generation), written in core-matrix layout: pieces[q * kPieceBytes + core_off(r, k)].
__global__ void k_dft_matrix(unsigned char* pieces, int P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kM * kK) return;
    const int r = i / kK, k = i % kK;
    const int blk = 2 * P;
    double a = 0.0;
    if (r / blk == k / blk) {
        const int rr = r % blk, kk = k % blk;
        const int kout = rr % P, jin = kk % P;
        const bool out_im = rr >= P, in_im = kk >= P;
        double s, c;  // W = e^{-2 pi i j k / P} = c - i s
        sincospi(2.0 * (double)((int64_t)jin * kout % P) / (double)P, &s, &c);
        // [re; im] out = [[c, s], [-s, c]] [re; im] in
        if (!out_im) a = in_im ? s : c;
        else a = in_im ? c : -s;
    }
    const __nv_bfloat16 h1 = __double2bfloat16(a);
    const double r1 = a - (double)__bfloat162float(h1);
    const __nv_bfloat16 h2 = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(h2);
    const __nv_bfloat16 h3 = __double2bfloat16(r2);
    const int off = core_off(r, k);
    *(__nv_bfloat16*)(pieces + off) = h1;
    *(__nv_bfloat16*)(pieces + kPieceBytes + off) = h2;
    *(__nv_bfloat16*)(pieces + 2 * kPieceBytes + off) = h3;
}

// tw4[j2 B1 + k1] = e^{-2 pi i j2 k1 / B} (four-step twiddles)
__global__ void k_dft_twiddles(float2* tw4, int B, int B1, int B2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const int j2 = i / B1, k1 = i % B1;
    double s, c;
    sincospi(2.0 * (double)((int64_t)j2 * k1 % B) / (double)B, &s, &c);
    tw4[i] = make_float2((float)c, (float)-s);
    (void)B2;
}

struct DftArgs {
    const float2* in;
    int64_t in_stride;     // per signal
    float2* out;
    int64_t out_stride;    // per signal
    const unsigned char* A;  // three bf16 pieces in core-matrix layout
    const float2* tw4;     // stage 2 twiddles (B entries)
    int32_t* status;       // set to 1 if a bounded wait gave up
    const float2* const* in_cols;  // optional per-column input base pointers (else strides)
    float2* const* out_cols;       // optional per-column output base pointers
    int B, B1, B2, R, P, copies, stage;  // stage 0: single (P = B); 1: four-step first; 2: second
    int64_t nvec, ngcols;
};

__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
    a = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(a);
    b = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b);
    c = __float2bfloat16_rn(r2);
}

__global__ void __launch_bounds__(kDftThreads, 1) k_dft_bf16x3(const DftArgs a) {
    static_assert(kDftThreads == 512 && kNT == 128, "epilogue maps 4 warpgroups to 4 x 32 columns");
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = sm;                      // 3 pieces of A
    unsigned char* sX = sm + 3 * kPieceBytes;    // 3 pieces of the column tile
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;

    // A: straight copy of the pre-laid-out pieces (16-byte vectors)
    for (int i = tid; i < 3 * kPieceBytes / 16; i += kDftThreads)
        ((uint4*)sA)[i] = __ldg((const uint4*)a.A + i);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kNT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    const int P = a.P, copies = a.copies, B = a.B, B1 = a.B1, B2 = a.B2, R = a.R;
    const int64_t ntiles = (a.ngcols + kNT - 1) / kNT;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
        const int64_t g0 = ti * kNT;
        // ---- gather the tile's input vectors into the three X pieces -----------------
        // GEMM column n holds vectors v = (g0 + n) copies + cc; K rows cc 2P + e (re) and
        // cc 2P + P + e (im) hold element e of vector cc.  One work item = 8 consecutive
        // elements of one vector (P >= 8): two 16-byte core rows (re and im) per piece.
        {
            const int chunks = P >> 3;
            for (int item = tid; item < kNT * 8; item += kDftThreads) {
                const int n = item % kNT, rest = item / kNT;
                const int cc = rest / chunks, e0 = (rest - cc * chunks) * 8;
                const int64_t v = (g0 + n) * copies + cc;
                float2 val[8];
                if (g0 + n < a.ngcols && v < a.nvec) {
                    if (a.stage == 0) {
                        const float2* cb = a.in_cols ? a.in_cols[v] : a.in + (v / R) * a.in_stride + (v % R) * B;
                        const float4* src = (const float4*)(cb + e0);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 f = src[q];
                            val[2 * q] = make_float2(f.x, f.y);
                            val[2 * q + 1] = make_float2(f.z, f.w);
                        }
                    } else if (a.stage == 1) {
                        const int64_t col = v / B2;
                        const int j2 = (int)(v - col * B2);
                        const float2* cb = a.in_cols ? a.in_cols[col] : a.in + (col / R) * a.in_stride + (col % R) * B;
#pragma unroll
                        for (int q = 0; q < 8; ++q) val[q] = cb[j2 + (int64_t)B2 * (e0 + q)];
                    } else {
                        const int64_t col = v / B1;
                        const int k1 = (int)(v - col * B1);
                        const float2* cb = a.in_cols ? a.in_cols[col] : a.in + (col / R) * a.in_stride + (col % R) * B;
                        const float4* src = (const float4*)(cb + (int64_t)k1 * B2 + e0);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 f = src[q];
                            val[2 * q] = make_float2(f.x, f.y);
                            val[2 * q + 1] = make_float2(f.z, f.w);
                        }
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float2 w = a.tw4[(e0 + q) * B1 + k1];
                            const float2 u = val[q];
                            val[q] = make_float2(u.x * w.x - u.y * w.y, u.x * w.y + u.y * w.x);
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) val[q] = make_float2(0.f, 0.f);
                }
                __align__(16) __nv_bfloat16 re[3][8], imv[3][8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    split3(val[q].x, re[0][q], re[1][q], re[2][q]);
                    split3(val[q].y, imv[0][q], imv[1][q], imv[2][q]);
                }
                const int ore = core_off(n, cc * 2 * P + e0), oim = core_off(n, cc * 2 * P + P + e0);
#pragma unroll
                for (int pc = 0; pc < 3; ++pc) {
                    *(uint4*)(sX + pc * kPieceBytes + ore) = *(const uint4*)re[pc];
                    *(uint4*)(sX + pc * kPieceBytes + oim) = *(const uint4*)imv[pc];
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- 8 K-steps x 6 products into the FP32 accumulator --------------------------
        if (tid == 0) {
            const uint32_t a0 = smem_u32(sA), x0 = smem_u32(sX);
            const int pa[6] = {0, 0, 1, 0, 1, 2}, px[6] = {0, 1, 0, 2, 1, 0};
            for (int ks = 0; ks < kK / 16; ++ks) {
                for (int q = 0; q < 6; ++q) {
                    const uint64_t ad = smem_desc(a0 + pa[q] * kPieceBytes + ks * 256);
                    const uint64_t bd = smem_desc(x0 + px[q] * kPieceBytes + ks * 256);
                    const uint32_t acc = (ks > 0 || q > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar)));
        }
        // ---- bounded wait for the accumulator -------------------------------------------
        uint32_t done = 0;
        for (uint32_t it = 0; it < kWaitLimit && !done; ++it) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                " selp.u32 %0, 1, 0, p;\n}"
                : "=r"(done)
                : "r"(smem_u32(&mbar)), "r"(phase));
        }
        phase ^= 1u;
        if (!__syncthreads_and(done)) {
            if (tid == 0) atomicExch(a.status, 1);
            ok = false;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- epilogue: TMEM rows -> shared stage (row stride kNT + 1) -> complex outputs -
        float* stg = (float*)sX;  // the X pieces are free once the MMAs completed
        {
            // warp w reads TMEM lanes 32 (w % 4) .. +31 (rows), columns 32 (w / 4) .. +31
            const int lg = warp & 3, wg = warp >> 2;
            const int row = lg * 32 + (tid & 31);
            for (int c0 = wg * 32; c0 < wg * 32 + 32; c0 += 16) {
                uint32_t d[16];
                const uint32_t ta = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
                      "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 16; ++j) stg[row * (kNT + 1) + c0 + j] = __uint_as_float(d[j]);
            }
        }
        __syncthreads();
        // output items (n, cc, k): stage 0 keeps k fastest (contiguous outputs), stages 1-2
        // keep n fastest (consecutive GEMM columns are consecutive output positions)
        for (int item = tid; item < kNT * 64; item += kDftThreads) {
            int n, cc, k;
            if (a.stage == 0) {
                k = item % P;
                const int rest = item / P;
                cc = rest % copies;
                n = rest / copies;
            } else {
                n = item % kNT;
                const int rest = item / kNT;
                cc = rest / P;
                k = rest - cc * P;
            }
            const int64_t g = g0 + n;
            const int64_t v = g * copies + cc;
            if (g >= a.ngcols || v >= a.nvec) continue;
            const float2 val = make_float2(stg[(cc * 2 * P + k) * (kNT + 1) + n],
                                           stg[(cc * 2 * P + P + k) * (kNT + 1) + n]);
            int64_t col, off;
            if (a.stage == 0) {
                col = v;
                off = k;
            } else if (a.stage == 1) {
                col = v / B2;
                const int j2 = (int)(v - col * B2);
                off = (int64_t)k * B2 + j2;
            } else {
                col = v / B1;
                const int k1 = (int)(v - col * B1);
                off = k1 + (int64_t)B1 * k;
            }
            float2* ob = a.out_cols ? a.out_cols[col] : a.out + (col / R) * a.out_stride + (col % R) * B;
            ob[off] = val;
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kNT));
}

}  // namespace

size_t dft_tc_matrix_bytes() { return 3 * (size_t)kPieceBytes; }

// Four-step factorisation B = B1 B2 with both factors in [8, 64] (single stage for B <= 64).
static void dft_factor(int B, int* B1, int* B2) {
    if (B <= 64) { *B1 = B; *B2 = 1; return; }
    int b1 = B / 8 < 64 ? B / 8 : 64;
    *B1 = b1;
    *B2 = B / b1;
}

int build_dft_tc_tables(int B, unsigned char* A1, unsigned char* A2, float2* tw4) {
    int B1, B2;
    dft_factor(B, &B1, &B2);
    k_dft_matrix<<<(kM * kK + 255) / 256, 256>>>(A1, B1);
    if (B2 > 1) {
        k_dft_matrix<<<(kM * kK + 255) / 256, 256>>>(A2, B2);
        k_dft_twiddles<<<(B + 255) / 256, 256>>>(tw4, B, B1, B2);
    }
    return check_cuda(cudaGetLastError());
}

int configure_dft_tc() {
    return check_cuda(cudaFuncSetAttribute(k_dft_bf16x3, cudaFuncAttributeMaxDynamicSharedMemorySize, kDftSmem));
}

// B-point DFTs of nsig x R columns of z (stride z_stride per signal) into y (stride
// y_stride), through the scratch u (same layout as z) for the four-step case.
int launch_dft_tc(const float2* z, int64_t z_stride, float2* u, float2* y, int64_t y_stride, int nsig,
                  int R, int B, const unsigned char* A1, const unsigned char* A2, const float2* tw4,
                  int32_t* status, int sm_count, cudaStream_t st, const float2* const* zcols,
                  float2* const* ucols, float2* const* ycols, int64_t ncols_override) {
    int B1, B2;
    dft_factor(B, &B1, &B2);
    DftArgs a;
    a.tw4 = tw4;
    a.status = status;
    a.B = B;
    a.B1 = B1;
    a.B2 = B2;
    a.R = R;
    const int64_t ncols = ncols_override > 0 ? ncols_override : (int64_t)nsig * R;
    auto run = [&](int stage, const float2* in, int64_t is, float2* out, int64_t os, int P,
                   const unsigned char* A, int64_t nvec, const float2* const* icols, float2* const* ocols) {
        a.stage = stage;
        a.in_cols = icols;
        a.out_cols = ocols;
        a.in = in;
        a.in_stride = is;
        a.out = out;
        a.out_stride = os;
        a.P = P;
        a.copies = 64 / P;
        a.A = A;
        a.nvec = nvec;
        a.ngcols = (nvec + a.copies - 1) / a.copies;
        const int64_t ntiles = (a.ngcols + kNT - 1) / kNT;
        const int grid = (int)(ntiles < sm_count ? ntiles : sm_count);
        k_dft_bf16x3<<<grid, kDftThreads, kDftSmem, st>>>(a);
        return check_cuda(cudaGetLastError());
    };
    if (B2 == 1) return run(0, z, z_stride, y, y_stride, B, A1, ncols, zcols, ycols);
    int rc = run(1, z, z_stride, u, z_stride, B1, A1, ncols * B2, zcols, ucols);
    if (rc) return rc;
    return run(2, u, z_stride, y, y_stride, B2, A2, ncols * B1, (const float2* const*)ucols, ycols);
}

}  // namespace sfft4
