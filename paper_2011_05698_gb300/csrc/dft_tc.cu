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
#include <string.h>

#include <vector>

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

// Polls the mbarrier at shared address `bar` for the completion of phase `parity`, at most
// `limit` times; returns 1 once it completed, 0 if the wait gave up.
__device__ __forceinline__ uint32_t mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t limit) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity));
    }
    return done;
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

// One (DFT matrix, stage) group of a launch: nvec input vectors of length P, 64 / P per GEMM
// column; columns come from per-column pointer tables or from (signal, round) strides.
struct DftGroup {
    const float2* in;
    int64_t in_stride;             // per signal (strided form)
    float2* out;
    int64_t out_stride;
    const float2* const* in_cols;  // optional per-column input base pointers
    float2* const* out_cols;       // optional per-column output base pointers
    const unsigned char* A;        // three bf16 pieces in core-matrix layout
    const float2* tw4;             // stage 2 twiddles (B entries)
    int B, B1, B2, R, P, copies, stage, pad;  // stage 0: single (P = B); 1, 2: four-step
    int lgP, lgC, lgB1, lgB2;      // log2 of P, copies, B1, B2 (all powers of two)
    int64_t nvec, ngcols, tile0;   // tile0: first tile of this group in the launch's list
};

constexpr int kDftMaxGroups = 12;

struct DftLaunch {
    DftGroup g[kDftMaxGroups];
    int32_t ngroups;
    int32_t* status;               // set to 1 if a bounded wait gave up
    int64_t ntiles;
};

__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
    a = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(a);
    b = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b);
    c = __float2bfloat16_rn(r2);
}

// Tile range [lo, hi) of the launch's tile list owned by CTA b of G (contiguous, so a CTA
// changes DFT matrix at most a few times).
__device__ __forceinline__ void cta_tiles(int64_t T, int64_t* lo, int64_t* hi) {
    *lo = (int64_t)blockIdx.x * T / gridDim.x;
    *hi = (int64_t)(blockIdx.x + 1) * T / gridDim.x;
}

__device__ __forceinline__ int group_of(const DftLaunch& L, int64_t ti) {
    int gi = 0;
    while (gi + 1 < L.ngroups && ti >= L.g[gi + 1].tile0) ++gi;
    return gi;
}

// Work item w of this thread: GEMM column n, vector cc within it, elements e0 .. e0 + 7.  A
// GEMM column holds vectors v = gc copies + cc; K rows cc 2P + e (re), cc 2P + P + e (im).
struct DftItem {
    int n, cc, e0;
};

__device__ __forceinline__ DftItem dft_item(const DftGroup& g, int item) {
    DftItem it;
    it.n = item & (kNT - 1);
    const int rest = item >> 7;  // kNT = 128
    it.cc = rest >> (g.lgP - 3);
    it.e0 = (rest & ((g.P >> 3) - 1)) << 3;
    return it;
}

// Gather the two work items of this thread for tile ti of group g into registers (group
// fields read once into registers before the loads).
__device__ __forceinline__ void dft_gather(const DftGroup& g, int64_t ti, int tid, float2 (&val)[2][8]) {
    const uint32_t g0 = (uint32_t)(ti - g.tile0) * kNT;
    const int stage = g.stage, lgB1 = g.lgB1, lgB2 = g.lgB2, lgC = g.lgC, lgP = g.lgP;
    const uint32_t b1m = (uint32_t)g.B1 - 1, b2m = (uint32_t)g.B2 - 1;
    const uint32_t ngc = (uint32_t)g.ngcols, nv = (uint32_t)g.nvec, Rr = (uint32_t)g.R;
    const float2* const* __restrict__ icols = g.in_cols;
    const float2* const ibase = g.in;
    const int64_t istr = g.in_stride, Bv = g.B;
    const float2* const __restrict__ tw4 = g.tw4;
    const int chm = (g.P >> 3) - 1;
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        const int item = tid + w * kDftThreads;
        const int n = item & (kNT - 1), rest = item >> 7;
        const int cc = rest >> (lgP - 3), e0 = (rest & chm) << 3;
        const uint32_t gc = g0 + n;
        const uint32_t v = (gc << lgC) + cc;
        if (gc < ngc && v < nv) {
            const uint32_t col = stage == 0 ? v : (stage == 1 ? (v >> lgB2) : (v >> lgB1));
            const float2* cb;
            if (icols) {
                cb = icols[col];
            } else {
                const uint32_t sg = col / Rr, r = col - sg * Rr;
                cb = ibase + (int64_t)sg * istr + (int64_t)r * Bv;
            }
            if (stage == 0) {
                const float4* src = (const float4*)(cb + e0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 f = __ldg(src + q);
                    val[w][2 * q] = make_float2(f.x, f.y);
                    val[w][2 * q + 1] = make_float2(f.z, f.w);
                }
            } else if (stage == 1) {
                const float2* p = cb + (v & b2m) + ((uint32_t)e0 << lgB2);
#pragma unroll
                for (int q = 0; q < 8; ++q) val[w][q] = __ldg(p + ((uint32_t)q << lgB2));
            } else {
                // stage 2 reads the stage-1 output written by the previous launch
                const uint32_t k1 = v & b1m;
                const float4* src = (const float4*)(cb + (k1 << lgB2) + e0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 f = src[q];
                    val[w][2 * q] = make_float2(f.x, f.y);
                    val[w][2 * q + 1] = make_float2(f.z, f.w);
                }
                const float2* tw = tw4 + ((uint32_t)e0 << lgB1) + k1;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float2 t = __ldg(tw + ((uint32_t)q << lgB1));
                    const float2 u = val[w][q];
                    val[w][q] = make_float2(u.x * t.x - u.y * t.y, u.x * t.y + u.y * t.x);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) val[w][q] = make_float2(0.f, 0.f);
        }
    }
}

// Split the gathered items into the three bf16 X pieces (core-matrix layout).
__device__ __forceinline__ void dft_store_x(const DftGroup& g, int tid, const float2 (&val)[2][8],
                                            unsigned char* sX) {
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        const DftItem it = dft_item(g, tid + w * kDftThreads);
        __align__(16) __nv_bfloat16 re[3][8], imv[3][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            split3(val[w][q].x, re[0][q], re[1][q], re[2][q]);
            split3(val[w][q].y, imv[0][q], imv[1][q], imv[2][q]);
        }
        const int kre = (it.cc << (g.lgP + 1)) + it.e0;
        const int ore = core_off(it.n, kre), oim = core_off(it.n, kre + g.P);
#pragma unroll
        for (int pc = 0; pc < 3; ++pc) {
            *(uint4*)(sX + pc * kPieceBytes + ore) = *(const uint4*)re[pc];
            *(uint4*)(sX + pc * kPieceBytes + oim) = *(const uint4*)imv[pc];
        }
    }
}

// Persistent CTAs over the tile list of up to kDftMaxGroups (matrix, stage) groups.  Per tile:
// the gathered registers are split into X, one thread issues the 8 K-steps x 6 products, the
// next tile's gather is issued while the MMAs run, then the accumulator goes through TMEM ->
// shared stage -> coalesced stores.
__global__ void __launch_bounds__(kDftThreads, 1) k_dft_bf16x3(const __grid_constant__ DftLaunch L) {
    static_assert(kDftThreads == 512 && kNT == 128, "epilogue maps 4 warpgroups to 4 x 32 columns");
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = sm;                      // 3 pieces of A
    unsigned char* sX = sm + 3 * kPieceBytes;    // 3 pieces of the column tile
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t abar;  // completion of the DFT matrix's bulk copy
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    int64_t t_lo, t_hi;
    cta_tiles(L.ntiles, &t_lo, &t_hi);
    if (t_lo >= t_hi) return;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kNT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&abar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    uint32_t phase = 0, aphase = 0;
    int cur = -1;  // group whose matrix is in sA
    float2 val[2][8];
    int gi = group_of(L, t_lo);
    dft_gather(L.g[gi], t_lo, tid, val);
    for (int64_t ti = t_lo; ti < t_hi; ++ti) {
        const DftGroup& g = L.g[gi];
        if (gi != cur) {
            // the previous tile's MMAs have completed, so A may be replaced: one thread
            // issues bulk copies of the three pieces (TMA), everyone waits on their bytes
            if (tid == 0) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&abar)),
                             "r"(3 * kPieceBytes));
#pragma unroll
                for (int pc = 0; pc < 3; ++pc)
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(sA + pc * kPieceBytes)),
                        "l"(g.A + pc * kPieceBytes), "r"(kPieceBytes), "r"(smem_u32(&abar))
                        : "memory");
            }
            cur = gi;
            dft_store_x(g, tid, val, sX);
            const uint32_t adone = mbar_wait_bounded(smem_u32(&abar), aphase, kWaitLimit);
            if (!__syncthreads_and(adone)) {
                // give up: report, then give the bulk copy still in flight one more bounded wait
                // before the CTA leaves (no MMA of this tile has been issued)
                if (tid == 0) atomicExch(L.status, 1);
                mbar_wait_bounded(smem_u32(&abar), aphase, kWaitLimit);
                break;
            }
            aphase ^= 1u;
        } else {
            dft_store_x(g, tid, val, sX);
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- 8 K-steps x 6 products into the FP32 accumulator --------------------------
        if (tid == 0) {
            // descriptors advance by (byte offset >> 4) in their start-address field
            const uint64_t da = smem_desc(smem_u32(sA)), dx = smem_desc(smem_u32(sX));
#pragma unroll
            for (int ks = 0; ks < kK / 16; ++ks) {
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const int pa = (q == 2 || q == 4) ? 1 : (q == 5 ? 2 : 0);  // a1x1 a1x2 a2x1 a1x3 a2x2 a3x1
                    const int px = (q == 1 || q == 4) ? 1 : (q == 3 ? 2 : 0);
                    const uint64_t ad = da + (uint64_t)((pa * kPieceBytes + ks * 256) >> 4);
                    const uint64_t bd = dx + (uint64_t)((px * kPieceBytes + ks * 256) >> 4);
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
        // ---- the next tile's gather is in flight while the MMAs run ---------------------
        const int gn = (ti + 1 < t_hi) ? group_of(L, ti + 1) : gi;
        if (ti + 1 < t_hi) dft_gather(L.g[gn], ti + 1, tid, val);
        // ---- bounded wait for the accumulator -------------------------------------------
        const uint32_t done = mbar_wait_bounded(smem_u32(&mbar), phase, kWaitLimit);
        if (!__syncthreads_and(done)) {
            // give up: report, then wait once more (bounded) for the commit of this tile's MMAs,
            // which still write the accumulator, before its TMEM columns are freed below.  If
            // that wait gives up too the columns are freed regardless: a CTA must not exit
            // holding tensor memory.
            if (tid == 0) atomicExch(L.status, 1);
            mbar_wait_bounded(smem_u32(&mbar), phase, kWaitLimit);
            break;
        }
        phase ^= 1u;
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
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        {
            // every group field the loop needs is read once into registers: the output stores
            // go through generic pointers, after which the parameter block would be re-read
            const uint32_t g0 = (uint32_t)(ti - g.tile0) * kNT;
            const int P = g.P, lgP = g.lgP, lgC = g.lgC, stage = g.stage;
            const int lgB1 = g.lgB1, lgB2 = g.lgB2;
            const uint32_t cm = (uint32_t)g.copies - 1, b1m = (uint32_t)g.B1 - 1, b2m = (uint32_t)g.B2 - 1;
            const uint32_t ngc = (uint32_t)g.ngcols, nv = (uint32_t)g.nvec, Rr = (uint32_t)g.R;
            float2* const* __restrict__ ocols = g.out_cols;
            float2* const obase = g.out;
            const int64_t ostr = g.out_stride, Bv = g.B;
            // output items (n, cc, k): stage 0 keeps k fastest (contiguous outputs), stages 1-2
            // keep n fastest (consecutive GEMM columns are consecutive output positions)
#pragma unroll 4
            for (int item = tid; item < kNT * 64; item += kDftThreads) {
                int n, cc, k;
                if (stage == 0) {
                    k = item & (P - 1);
                    const int rest = item >> lgP;
                    cc = rest & cm;
                    n = rest >> lgC;
                } else {
                    n = item & (kNT - 1);
                    const int rest = item >> 7;
                    cc = rest >> lgP;
                    k = rest & (P - 1);
                }
                const uint32_t gc = g0 + n;
                const uint32_t v = (gc << lgC) + cc;
                if (gc >= ngc || v >= nv) continue;
                const int kr = (cc << (lgP + 1)) + k;
                const float2 o = make_float2(stg[kr * (kNT + 1) + n], stg[(kr + P) * (kNT + 1) + n]);
                uint32_t col, off;
                if (stage == 0) {
                    col = v;
                    off = k;
                } else if (stage == 1) {
                    col = v >> lgB2;
                    off = ((uint32_t)k << lgB2) + (v & b2m);
                } else {
                    col = v >> lgB1;
                    off = (v & b1m) + ((uint32_t)k << lgB1);
                }
                float2* ob;
                if (ocols) {
                    ob = ocols[col];
                } else {
                    const uint32_t sg = col / Rr, r = col - sg * Rr;
                    ob = obase + (int64_t)sg * ostr + (int64_t)r * Bv;
                }
                ob[off] = o;
            }
        }
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        gi = gn;
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

namespace {

int ilog2i(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

DftGroup make_group(int stage, int B, int P, const unsigned char* A, const float2* tw4, int64_t nvec) {
    DftGroup g;
    memset(&g, 0, sizeof(g));
    int B1, B2;
    dft_factor(B, &B1, &B2);
    g.B = B;
    g.B1 = B1;
    g.B2 = B2;
    g.R = 1;
    g.P = P;
    g.copies = 64 / P;
    g.stage = stage;
    g.lgP = ilog2i(P);
    g.lgC = ilog2i(g.copies);
    g.lgB1 = ilog2i(B1);
    g.lgB2 = ilog2i(B2);
    g.A = A;
    g.tw4 = tw4;
    g.nvec = nvec;
    g.ngcols = (nvec + g.copies - 1) / g.copies;
    return g;
}

// One launch over up to kDftMaxGroups groups (tiles numbered group after group).
int launch_groups(std::vector<DftGroup>& gs, int32_t* status, int sm_count, cudaStream_t st) {
    size_t i0 = 0;
    while (i0 < gs.size()) {
        DftLaunch L;
        memset(&L, 0, sizeof(L));
        L.status = status;
        int64_t T = 0;
        int n = 0;
        for (; n < kDftMaxGroups && i0 + n < gs.size(); ++n) {
            DftGroup g = gs[i0 + n];
            g.tile0 = T;
            T += (g.ngcols + kNT - 1) / kNT;
            L.g[n] = g;
        }
        L.ngroups = n;
        L.ntiles = T;
        i0 += n;
        if (T == 0) continue;
        const int grid = (int)(T < sm_count ? T : sm_count);
        k_dft_bf16x3<<<grid, kDftThreads, kDftSmem, st>>>(L);
        int rc = check_cuda(cudaGetLastError());
        if (rc) return rc;
    }
    return SFFT4_OK;
}

}  // namespace

// B-point DFTs of nsig x R columns of z (stride z_stride per signal) into y (stride
// y_stride), through the scratch u (same layout as z) for the four-step case.
int launch_dft_tc(const float2* z, int64_t z_stride, float2* u, int64_t u_stride, float2* y, int64_t y_stride, int nsig,
                  int R, int B, const unsigned char* A1, const unsigned char* A2, const float2* tw4,
                  int32_t* status, int sm_count, cudaStream_t st) {
    int B1, B2;
    dft_factor(B, &B1, &B2);
    const int64_t ncols = (int64_t)nsig * R;
    std::vector<DftGroup> gs(1);
    if (B2 == 1) {
        gs[0] = make_group(0, B, B, A1, tw4, ncols);
        gs[0].in = z, gs[0].in_stride = z_stride, gs[0].out = y, gs[0].out_stride = y_stride, gs[0].R = R;
        return launch_groups(gs, status, sm_count, st);
    }
    gs[0] = make_group(1, B, B1, A1, tw4, ncols * B2);
    gs[0].in = z, gs[0].in_stride = z_stride, gs[0].out = u, gs[0].out_stride = u_stride, gs[0].R = R;
    int rc = launch_groups(gs, status, sm_count, st);
    if (rc) return rc;
    gs[0] = make_group(2, B, B2, A2, tw4, ncols * B1);
    gs[0].in = u, gs[0].in_stride = u_stride, gs[0].out = y, gs[0].out_stride = y_stride, gs[0].R = R;
    return launch_groups(gs, status, sm_count, st);
}

// DFTs of every iteration of a uniform batch at once (the signal-major fold has made all
// their folded arrays): one launch for the single-stage and first four-step stages of every
// iteration, one for the second stages, instead of one or two launches per iteration.
int launch_dft_tc_strided(const DftStrided* sets, int nsets, int32_t* status, int sm_count, cudaStream_t st) {
    std::vector<DftGroup> a, b;
    for (int i = 0; i < nsets; ++i) {
        const DftStrided& c = sets[i];
        int B1, B2;
        dft_factor(c.B, &B1, &B2);
        const int64_t ncols = (int64_t)c.nsig * c.R;
        if (B2 == 1) {
            DftGroup g = make_group(0, c.B, c.B, c.A1, c.tw4, ncols);
            g.in = c.z, g.in_stride = c.z_stride, g.out = c.y, g.out_stride = c.y_stride, g.R = c.R;
            a.push_back(g);
        } else {
            DftGroup g1 = make_group(1, c.B, B1, c.A1, c.tw4, ncols * B2);
            g1.in = c.z, g1.in_stride = c.z_stride, g1.out = c.u, g1.out_stride = c.u_stride, g1.R = c.R;
            a.push_back(g1);
            DftGroup g2 = make_group(2, c.B, B2, c.A2, c.tw4, ncols * B1);
            g2.in = c.u, g2.in_stride = c.u_stride, g2.out = c.y, g2.out_stride = c.y_stride, g2.R = c.R;
            b.push_back(g2);
        }
    }
    int rc = launch_groups(a, status, sm_count, st);
    if (!rc) rc = launch_groups(b, status, sm_count, st);
    return rc;
}

// DFTs of column sets of several bucket counts (a level of a batch of uneven signals): one
// launch for the single-stage and first four-step stages of every set, one for the second.
int launch_dft_tc_sets(const DftColSet* sets, int nsets, int32_t* status, int sm_count, cudaStream_t st) {
    std::vector<DftGroup> a, b;
    for (int i = 0; i < nsets; ++i) {
        const DftColSet& c = sets[i];
        int B1, B2;
        dft_factor(c.B, &B1, &B2);
        if (B2 == 1) {
            DftGroup g = make_group(0, c.B, c.B, c.A1, c.tw4, c.ncols);
            g.in_cols = c.zcols, g.out_cols = c.ycols;
            a.push_back(g);
        } else {
            DftGroup g1 = make_group(1, c.B, B1, c.A1, c.tw4, c.ncols * B2);
            g1.in_cols = c.zcols, g1.out_cols = c.ucols;
            a.push_back(g1);
            DftGroup g2 = make_group(2, c.B, B2, c.A2, c.tw4, c.ncols * B1);
            g2.in_cols = (const float2* const*)c.ucols, g2.out_cols = c.ycols;
            b.push_back(g2);
        }
    }
    int rc = launch_groups(a, status, sm_count, st);
    if (!rc) rc = launch_groups(b, status, sm_count, st);
    return rc;
}

int dft_tc_launches(const int* Bs, int nsets) {
    int na = 0, nb = 0;
    for (int i = 0; i < nsets; ++i) {
        int B1, B2;
        dft_factor(Bs[i], &B1, &B2);
        ++na;
        if (B2 > 1) ++nb;
    }
    return (na + kDftMaxGroups - 1) / kDftMaxGroups + (nb + kDftMaxGroups - 1) / kDftMaxGroups;
}

}  // namespace sfft4
