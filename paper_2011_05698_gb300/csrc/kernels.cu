// sm_103a kernels of the sFFT4.0 hot path and the execute entry points.
//
//   k_window_*  flat window G (FP64 generation, FP32 copy) and its spectrum G'^ (Eq. 9-10)
//   k_fold      permuted int64-exact gather x[(sigma t + a) mod N], window multiply and fold
//               into B slots for every round of one iteration (Lemma 1, steps P0-P3)
//   k_fft       B-point DFT of every (signal, round) column, FP32 radix-2 (Lemma 1, P3)
//   k_decode    bucket update (Section 3.1), large-bucket selection, multiscale location
//               with votes (Section 3.2, Eq. 15-19), median estimation (Eq. 14) and merge
//   k_finalize  top-K by |v| and sort by frequency
//
// Determinism: every reduction has a fixed order (per-thread sequential sums, fixed-order
// sums over copies, radix-2 butterflies), and the bucket update accumulates in int64
// fixed point with order-independent integer atomics, so repeated runs are bit-identical.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include <cooperative_groups.h>

#include "sfft4_internal.cuh"

namespace cg = cooperative_groups;

namespace sfft4 {

// ----------------------------------------------------------------- small helpers ----
__device__ __forceinline__ float2 ld_stream(const float2* p) {
    float2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

// (cos, sin) of 2 pi r / 2^n for 0 <= r < 2^n, with exactly representable sincospif
// arguments: r = rh 2^12 + rl, angle = 2 pi rh / 2^(n-12) + 2 pi rl / 2^n.
__device__ __forceinline__ float2 cis_2pi_frac(uint64_t r, int n) {
    // r < 2^n <= 2^30: 32-bit conversions (64-bit integer conversions run at the FP64 rate)
    const uint32_t r32 = (uint32_t)r;
    float s, c;
    if (n <= 24) {
        sincospif(ldexpf((float)r32, 1 - n), &s, &c);
        return make_float2(c, s);
    }
    float sa, ca, sb, cb;
    sincospif(ldexpf((float)(r32 >> 12), 13 - n), &sa, &ca);
    sincospif(ldexpf((float)(r32 & 4095u), 1 - n), &sb, &cb);
    return make_float2(ca * cb - sa * sb, sa * cb + ca * sb);
}

// rint(x) as int64 (round half to even, as __float2ll_rn) in float adds: for |x| <= 2^45,
// x = h 2^23 + d with h = rint(x / 2^23) and d exact (one fmaf, |d| <= 2^22), and
// rint(x) = h 2^23 + rint(d) because h 2^23 is an even integer.  Both roundings add
// 1.5 2^23: a float in [2^23, 2^24] has unit spacing, so the sum is rounded to the nearest
// integer (half to even) and its low mantissa bits hold that integer plus 2^22.  This keeps
// the float-to-int conversion unit (a few lanes per clock) out of the update's inner loop.
// Out-of-range cases call the 64-bit conversion in a separate function, so that the
// compiler cannot if-convert it into every lane.
__device__ __noinline__ long long f2ll_rn_wide(float x) { return __float2ll_rn(x); }
__device__ __noinline__ float ll2f_rn_wide(long long v) { return __ll2float_rn(v); }

__device__ __forceinline__ long long f2ll_rn(float x) {
    if (!(fabsf(x) <= 0x1p45f)) return f2ll_rn_wide(x);
    constexpr float M = 12582912.f;  // 1.5 2^23
    const float th = __fadd_rn(x * 0x1p-23f, M);
    const int h = __float_as_int(th) - 0x4B400000;
    const float d = fmaf(-__fsub_rn(th, M), 0x1p23f, x);
    const int r = __float_as_int(__fadd_rn(d, M)) - 0x4B400000;
    return ((long long)h << 23) + r;
}

// The float nearest to v (ties to even, as __ll2float_rn): for |v| < 2^48, v = h 2^24 + l
// with 0 <= l < 2^24, both exact in float, and one rounding in fmaf.
__device__ __forceinline__ float ll2f_rn(long long v) {
    if (v >= (1ll << 48) || v <= -(1ll << 48)) return ll2f_rn_wide(v);
    return fmaf((float)(int)(v >> 24), 0x1p24f, (float)(int)(v & 0xFFFFFF));
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ----------------------------------------------------------------- window -----------
__global__ void k_window_time(double* g64, int64_t h, int64_t N, int64_t M, double s_t) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > 2 * h) return;
    int64_t j = i - h;
    double x = (double)j / s_t;
    double g = exp(-0.5 * x * x);
    double D;
    if (j == 0) {
        D = (double)(2 * M + 1);
    } else {
        // Dirichlet kernel of the box |k| <= M: sin(pi (2M+1) j / N) / sin(pi j / N),
        // integer arguments reduced mod 2N first
        int64_t twoN = 2 * N;
        int64_t r1 = (((2 * M + 1) * j) % twoN + twoN) % twoN;
        int64_t r2 = ((j % twoN) + twoN) % twoN;
        D = sinpi((double)r1 / (double)N) / sinpi((double)r2 / (double)N);
    }
    g64[i] = g * D;
}

__global__ void k_window_norm(const double* g64, int64_t w, float* G32) {
    __shared__ double red[1024];
    double s = 0;
    for (int64_t i = threadIdx.x; i < w; i += blockDim.x) s += g64[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    double tot = red[0];
    for (int64_t i = threadIdx.x; i < w; i += blockDim.x) G32[i] = (float)(g64[i] / tot);
}

// G'^_k = sum_{j=-h..h} G_j cos(2 pi k j / N), one warp per k, Kahan-compensated FP32
// terms per lane, lanes combined in FP64.
__global__ void k_window_spectrum(const float* G32, int64_t h, int64_t N, int n, int64_t nk,
                                  float* Ghat) {
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= nk) return;
    uint64_t k = (uint64_t)warp;
    float sum = 0.f, comp = 0.f;
    for (int64_t i = lane; i <= 2 * h; i += 32) {
        int64_t j = i - h;
        uint64_t r = (k * (uint64_t)j) & (uint64_t)(N - 1);
        float term = G32[i] * cis_2pi_frac(r, n).x;
        float yk = term - comp;
        float t = sum + yk;
        comp = (t - sum) - yk;
        sum = t;
    }
    double tot = (double)sum - (double)comp;
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
    if (lane == 0) Ghat[k] = (float)tot;
}

__global__ void k_twiddles(float2* tw, int B) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B / 2) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)B, &s, &c);
    tw[k] = make_float2((float)c, (float)-s);
}

int build_window_tables(sfft4_plan_s* p, Window* w, double delta) {
    int64_t N = p->N, L = w->L, h = w->h, wlen = 2 * h + 1;
    double s_t = 0.0;
    if (window_halfwidth(w->B, delta, &s_t) != h) return SFFT4_EINVAL;  // the planner's h
    int64_t M = (3 * L) / 4;
    double* g64 = nullptr;
    int rc = check_cuda(cudaMalloc(&g64, wlen * sizeof(double)));
    if (rc) return rc;
    int64_t nk = (3 * L) / 2 + 1;
    rc = check_cuda(cudaMalloc(&w->G, wlen * sizeof(float)));
    if (!rc) rc = check_cuda(cudaMalloc(&w->Ghat, nk * sizeof(float)));
    if (!rc) rc = check_cuda(cudaMalloc(&w->tw, (w->B / 2) * sizeof(float2)));
    if (rc) { cudaFree(g64); return rc; }
    k_window_time<<<(unsigned)((wlen + 255) / 256), 256>>>(g64, h, N, M, s_t);
    k_window_norm<<<1, 1024>>>(g64, wlen, w->G);
    k_window_spectrum<<<(unsigned)((nk * 32 + 255) / 256), 256>>>(w->G, h, N, p->n, nk, w->Ghat);
    k_twiddles<<<(w->B / 2 + 255) / 256, 256>>>(w->tw, w->B);
    rc = check_cuda(cudaGetLastError());
    if (!rc) rc = check_cuda(cudaDeviceSynchronize());
    cudaFree(g64);
    return rc;
}

// ----------------------------------------------------------------- fold -------------

// gathers in flight per thread: with fold groups of at most 3 rounds, 4 measured 1.9 % faster
// than 8 (with groups of 6 rounds 8 had been 1.2 % faster than 4); 16 spills
constexpr int kFoldUnroll = 4;

// One CTA = (signal, slice of Wj residues mod B).  Thread (jj, p) owns the samples
// t = rho + m' B with rho = slice Wj + jj and m' = p (mod P), so its fold slot for round s,
// (t - tau_s) mod B, is fixed: it accumulates in registers, then the P copies of each slot
// are summed in a fixed order.  Each x sample is loaded once for all rounds whose window
// covers it; its window coefficient for round s, G[t - tau_s + h], is loaded from the table
// beside it (the 32 lanes of a warp hold consecutive residues, so the coefficient loads of a
// warp are contiguous).  The copies of every round are summed after one barrier.  Index
// arithmetic is exact in 32 bits: N = 2^n divides 2^32, so (sigma t + a) mod N is the low n
// bits of the wrapped 32-bit value.  red: shared memory of RG x blockDim.x float2.
template <int RG>
__device__ __forceinline__ void fold_body(const FoldArgs& a, int slice, int64_t signal_index,
                                          const float2* __restrict__ x, float2* zsig, float2* red) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int Wj = a.Wj, B = a.B;
    const int P = a.g.P;
    const bool active = tid < Wj * P;  // a launch may carry more threads than this job uses
    const int jj = tid % Wj, p = tid / Wj;
    const int rho0 = slice * Wj;
    uint32_t sigma, aoff;
    {
        // the same draw in every thread (block-uniform, no barrier needed)
        uint64_t s, o;
        permutation_draw(a.seed, (uint64_t)signal_index, (uint64_t)a.m, a.N, &s, &o);
        sigma = (uint32_t)s;
        aoff = (uint32_t)o;
    }
    const uint32_t mask = (uint32_t)(a.N - 1);
    const int PB = P * B;
    const int rho = rho0 + jj + p * B;  // residue mod P B
    const uint32_t step = sigma * (uint32_t)PB;
    const float* __restrict__ G = a.G;
    float2 acc[RG];
#pragma unroll
    for (int s = 0; s < RG; ++s) acc[s] = make_float2(0.f, 0.f);

    for (int sg = 0; active && sg < a.g.nseg; ++sg) {
        const int t0 = (int)a.g.t0[sg], t1 = (int)a.g.t1[sg];
        const uint32_t rm = a.g.mask[sg];
        int d = (rho - t0) % PB;
        if (d < 0) d += PB;
        const int t = t0 + d;
        if (t >= t1) continue;
        const int cnt = (t1 - t + PB - 1) / PB;
        uint32_t idx = sigma * (uint32_t)t + aoff;
        const int gi0 = t + a.h;  // G index of sample k of round s: gi0 + k P B - tau_s
        for (int k = 0; k < cnt; k += kFoldUnroll) {
            float2 v[kFoldUnroll];
#pragma unroll
            for (int u = 0; u < kFoldUnroll; ++u) {
                v[u] = (k + u < cnt) ? ld_stream(x + (idx & mask)) : make_float2(0.f, 0.f);
                idx += step;
            }
#pragma unroll
            for (int u = 0; u < kFoldUnroll; ++u) {
                if (k + u < cnt) {
#pragma unroll
                    for (int s = 0; s < RG; ++s) {
                        if ((rm >> s) & 1u) {
                            const float gw = __ldg(G + (gi0 + (k + u) * PB - a.tau[s]));
                            acc[s].x = fmaf(gw, v[u].x, acc[s].x);
                            acc[s].y = fmaf(gw, v[u].y, acc[s].y);
                        }
                    }
                }
            }
        }
    }
    // the P copies of each (round, slot), summed in copy order 0 .. P-1
#pragma unroll
    for (int s = 0; s < RG; ++s)
        if (s < a.g.nr) red[s * T + tid] = acc[s];
    __syncthreads();
    for (int e = tid; e < a.g.nr * Wj; e += T) {
        const int s = e / Wj, j = e - s * Wj;
        const float2* rs = red + s * T + j;
        float2 sum = rs[0];
        for (int pp = 1; pp < P; ++pp) {
            const float2 o = rs[pp * Wj];
            sum.x += o.x;
            sum.y += o.y;
        }
        int slot = (rho0 + j - a.tau[s]) % B;
        if (slot < 0) slot += B;
        zsig[(int64_t)(a.g.r0 + s) * B + slot] = sum;
    }
}

template <int RG>
__global__ void __launch_bounds__(512, 2) k_fold(const FoldArgs a) {
    extern __shared__ float2 red[];  // [RG][blockDim.x]
    const int sig = blockIdx.y;
    fold_body<RG>(a, blockIdx.x, (int64_t)a.signal0 + sig, a.x + (int64_t)sig * a.x_stride,
                  a.z + (int64_t)sig * a.z_stride, red);
}

// Tile queue of a batch of signals with different N and K: CTA b takes tile tiles[b] = (job,
// residue slice) of one level; the job (a FoldArgs with the signal's own z block in z and its
// batch index in signal0) is copied to shared memory first.  x of signal s is xptrs[s].

template <int RG>
__global__ void __launch_bounds__(512, 2) k_fold_multi(const FoldArgs* __restrict__ jobs,
                                                       const FoldTile* __restrict__ tiles,
                                                       const float2* const* __restrict__ xptrs) {
    extern __shared__ float2 red[];  // [RG][blockDim.x]
    __shared__ __align__(16) FoldArgs sa;
    const FoldTile t = tiles[blockIdx.x];
    for (int i = threadIdx.x; i < (int)(sizeof(FoldArgs) / 4); i += blockDim.x)
        ((uint32_t*)&sa)[i] = ((const uint32_t*)(jobs + t.job))[i];
    __syncthreads();
    fold_body<RG>(sa, t.slice, sa.signal0, xptrs[sa.signal0], sa.z, red);
}

// Signal-major fold of a uniform batch: CTA b folds tile b mod ntiles of signal b / ntiles,
// the tiles of every (iteration, fold group) of one signal adjacent in the grid.  The CTAs
// resident at a time then gather from few signals, and a 32-byte sector that the permutations
// of several iterations draw from is read from DRAM once and hit in L2 after that; in
// iteration order every iteration re-reads it from DRAM.  The job arguments stay in the
// parameter space (indexed by a block-uniform job number).
template <int RG>
__global__ void __launch_bounds__(512, 2) k_fold_sig(const __grid_constant__ SigFoldLaunch L) {
    extern __shared__ float2 red[];  // [RG][blockDim.x]
    const int sig = blockIdx.x / L.ntiles;
    const int ti = blockIdx.x - sig * L.ntiles;
    int j = 0;
    while (j + 1 < L.njobs && ti >= L.start[j + 1]) ++j;
    const FoldArgs& a = L.jobs[j];
    fold_body<RG>(a, ti - L.start[j], (int64_t)a.signal0 + sig, L.x + (int64_t)sig * L.x_stride,
                  a.z + (int64_t)sig * a.z_stride, red);
}

// ----------------------------------------------------------------- FFT --------------
// Radix-2 decimation-in-time B-point DFT (unnormalised, e^{-2 pi i b j / B}) of
// `cpc` columns per CTA in shared memory; column c = signal * R + round.
__global__ void k_fft(const float2* __restrict__ z, float2* __restrict__ y, int B, int logB,
                      const float2* __restrict__ tw, int64_t z_stride, int64_t y_stride, int R,
                      int cpc, int ncols, const float2* const* zcols, float2* const* ycols) {
    extern __shared__ float2 sm[];
    const int tid = threadIdx.x, T = blockDim.x;
    const int c0 = blockIdx.x * cpc;
    const int ncol = min(cpc, ncols - c0);
    for (int i = tid; i < ncol * B; i += T) {
        int c = i >> logB, e = i & (B - 1);
        int col = c0 + c;
        const float2* zc = zcols ? zcols[col] : z + (int64_t)(col / R) * z_stride + (int64_t)(col % R) * B;
        sm[c * B + (__brev((unsigned)e) >> (32 - logB))] = zc[e];
    }
    __syncthreads();
    for (int ls = 0; ls < logB; ++ls) {
        const int hs = 1 << ls;
        for (int bf = tid; bf < ncol * (B >> 1); bf += T) {
            int c = bf >> (logB - 1), k = bf & ((B >> 1) - 1);
            int pos = k & (hs - 1), grp = k >> ls;
            int i0 = c * B + grp * 2 * hs + pos, i1 = i0 + hs;
            float2 w = tw[pos << (logB - 1 - ls)];
            float2 a0 = sm[i0], b0 = sm[i1];
            float2 bw = cmul(b0, w);
            sm[i0] = make_float2(a0.x + bw.x, a0.y + bw.y);
            sm[i1] = make_float2(a0.x - bw.x, a0.y - bw.y);
        }
        __syncthreads();
    }
    for (int i = tid; i < ncol * B; i += T) {
        int c = i >> logB, e = i & (B - 1);
        int col = c0 + c;
        float2* yc = ycols ? ycols[col] : y + (int64_t)(col / R) * y_stride + (int64_t)(col % R) * B;
        yc[e] = sm[c * B + e];
    }
}

// ----------------------------------------------------------------- block helpers ----
// Exclusive scan of per-thread counts over the block (up to 1024 threads); returns this
// thread's offset and writes the total to *total (all threads).
__device__ int block_exscan(int v, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int ws = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
        int wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_sums[lane] = wi - ws;
        if (lane == 31) warp_sums[32] = wi;
    }
    __syncthreads();
    int res = warp_sums[wid] + inc - v;
    *total = warp_sums[32];
    __syncthreads();
    return res;
}

__device__ int block_count(int v, int* slot) {
    int w = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) atomicAdd(slot, w);
    __syncthreads();
    int r = *slot;
    __syncthreads();
    if (threadIdx.x == 0) *slot = 0;
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint32_t hash_slot(int32_t f, int Hlog) {
    return ((uint32_t)f * 2654435761u) >> (32 - Hlog);
}

__device__ int32_t hash_find(const int32_t* keys, const int32_t* vals, int Hlog, int32_t f) {
    const uint32_t msk = (1u << Hlog) - 1;
    uint32_t s = hash_slot(f, Hlog);
    for (uint32_t probe = 0; probe <= msk; ++probe) {
        int32_t k = keys[s];
        if (k == f) return vals[s];
        if (k == -1) return -1;
        s = (s + 1) & msk;
    }
    return -1;
}

__device__ void hash_insert(int32_t* keys, int32_t* vals, int Hlog, int32_t f, int32_t idx) {
    const uint32_t msk = (1u << Hlog) - 1;
    uint32_t s = hash_slot(f, Hlog);
    for (uint32_t probe = 0; probe <= msk; ++probe) {
        int32_t prev = atomicCAS(&keys[s], -1, f);
        if (prev == -1) {
            vals[s] = idx;
            return;
        }
        s = (s + 1) & msk;
    }
}

// ----------------------------------------------------------------- decode -----------
constexpr int kUpdRounds = 4;  // rounds per pass of the gather update (int64 accumulators in registers)
// Largest B updated in gather form: with many found entries per bucket (small B) the gather
// avoids conflicting atomics; with few (B >= 1024) the scatter's single pass over the found
// set is shorter (phase timing on a GB300: 28 vs 41 us at B = 2048, 34 vs 40 us at B = 256).
constexpr int kGatherMaxB = 512;
// Dynamic shared memory of k_decode for B buckets: 26 B bytes of per-bucket arrays, and at
// least 108 KB for the update (staged found entries, 24 B each, or accumulator copies).  Two
// 512-thread CTAs fit on an SM.
__host__ __device__ inline size_t decode_tables_off(int B) { return (26 * (size_t)B + 15) & ~(size_t)15; }
__host__ __device__ inline size_t decode_smem(int B) {
    // the location's block-centre and region-shift tables (at most 63 block levels x 32 blocks
    // x 8 bytes) follow the per-bucket arrays
    const size_t base = decode_tables_off(B) + (size_t)(kMaxRounds - 1) * 32 * 8;
    const size_t upd = 108 * 1024;
    return base > upd ? base : upd;
}


// Median of v[0..R-1] (R <= RMAX): mean of the two middle values for even R (Eq. 14
// over rounds, reading R12).  RMAX = 16 sorts a fully unrolled bitonic network in registers
// (entries r >= R padded with +inf); larger RMAX falls back to an insertion sort.
template <int RMAX>
__device__ __forceinline__ float median_of(float (&v)[RMAX], int R) {
    if (RMAX <= 16) {
#pragma unroll
        for (int i = 0; i < RMAX; ++i)
            if (i >= R) v[i] = __int_as_float(0x7f800000);
#pragma unroll
        for (int k = 2; k <= RMAX; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
                for (int i = 0; i < RMAX; ++i) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const float lo = fminf(v[i], v[ixj]), hi = fmaxf(v[i], v[ixj]);
                        const bool up = (i & k) == 0;
                        v[i] = up ? lo : hi;
                        v[ixj] = up ? hi : lo;
                    }
                }
            }
        }
    } else {
        for (int i = 1; i < R; ++i) {
            float x = v[i];
            int j = i - 1;
            while (j >= 0 && v[j] > x) {
                v[j + 1] = v[j];
                --j;
            }
            v[j + 1] = x;
        }
    }
    float lo = 0.f, hi = 0.f;
#pragma unroll
    for (int i = 0; i < RMAX; ++i) {
        if (i == (R - 1) / 2) lo = v[i];
        if (i == R / 2) hi = v[i];
    }
    return (R & 1) ? hi : 0.5f * (lo + hi);
}

__device__ __forceinline__ uint32_t phase_fixed(float2 ys, float2 y0) {
    const float cr = ys.x * y0.x + ys.y * y0.y;
    const float cim = ys.y * y0.x - ys.x * y0.y;
    const float turns = atan2f(cim, cr) * 0.15915494309189535f;
    return (uint32_t)f2ll_rn(turns * 4294967296.0f);
}

// Phase of ys conj(y0) in 2^-32 turns from FP64 products and atan2 (the final level of the
// two-round location, whose integers are 2^(32-n) units apart).
__device__ __noinline__ uint32_t phase_fixed64(float2 ys, float2 y0) {
    const double cr = (double)ys.x * y0.x + (double)ys.y * y0.y;
    const double cim = (double)ys.y * y0.x - (double)ys.x * y0.y;
    const double turns = atan2(cim, cr) * 0.15915494309189533577;
    return (uint32_t)llrint(turns * 4294967296.0);
}

// Radix select over 32-bit keys held one chunk per thread: returns the value T of the
// n-th largest key (1 <= n <= count) by four passes over 8-bit digits, most significant
// first.  hist must hold 256 ints of shared memory; all threads of the block call it.
__device__ uint32_t block_radix_select(const float* key, int b_lo, int b_hi, int E, int n, int* hist,
                                       int* s_bcast) {
    // hist holds two 256-bin histograms and s_bcast two (digit, rank) pairs, used by
    // alternate passes: a pass counts into one histogram while the other is cleared for the
    // next, so each pass needs two barriers
    uint32_t prefix = 0, pmask = 0;
    int rank = n;  // rank of the wanted key among keys matching the prefix (1 = largest)
    for (int i = threadIdx.x; i < 512; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int d = 3; d >= 0; --d) {
        int* H = hist + 256 * (d & 1);
        int* Hn = hist + 256 * ((d & 1) ^ 1);
        int* bc = s_bcast + 2 * (d & 1);
        // warp-aggregated: lanes holding the same digit add once (keys cluster in a few
        // exponent bins, so plain atomics would serialise on those bins); E, the chunk length,
        // is the same in every thread, so all lanes take part in each match
        for (int e = 0; e < E; ++e) {
            const int b = b_lo + e;
            int digit = 256;
            if (b < b_hi) {
                const uint32_t k = __float_as_uint(key[b]);
                if ((k & pmask) == prefix) digit = (int)((k >> (8 * d)) & 255u);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, digit);
            if (digit < 256 && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1))
                atomicAdd(&H[digit], __popc(peers));
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // suffix sums from the top digit down: lane owns digits [248 - 8 lane, 255 - 8 lane]
            const int lane = threadIdx.x;
            int loc[8], tot = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) { loc[q] = H[255 - 8 * lane - q]; tot += loc[q]; }
            int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            int before = incl - tot;  // keys with a larger digit than this lane's range
            if (before < rank && rank <= incl) {
                int c = before;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (c < rank && rank <= c + loc[q]) {
                        bc[0] = 255 - 8 * lane - q;
                        bc[1] = rank - c;
                    }
                    c += loc[q];
                }
            }
        } else {
            for (int i = threadIdx.x - 32; i < 256; i += blockDim.x - 32) Hn[i] = 0;
        }
        __syncthreads();
        prefix |= (uint32_t)bc[0] << (8 * d);
        pmask |= 255u << (8 * d);
        rank = bc[1];
    }
    __syncthreads();
    return prefix;
}

// Barrier of the CTAs that decode one signal: the block itself, or (csize > 1) the thread-block
// cluster, after making this block's global writes (bucket updates) visible to the others.
__device__ __forceinline__ void decode_sync(int csize) {
    if (csize > 1) {
        __threadfence();
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

// Contiguous share [lo, hi) of n items of rank r among c ranks.
__device__ __forceinline__ void rank_share(int n, int r, int c, int* lo, int* hi) {
    *lo = (int)((int64_t)n * r / c);
    *hi = (int)((int64_t)n * (r + 1) / c);
}

// One CTA per signal, or a cluster of csize CTAs (rank crank) per signal: update the bucket
// arrays by the found set, select the large buckets, locate each candidate by the multiscale
// method, vote, estimate and merge.  All modular arithmetic is exact in 32 bits (N = 2^n
// divides 2^32).  RMAX bounds the rounds R of the iteration (16, or 64 for extreme (l, q)).
// In a cluster every rank stages the found set and selects the candidates itself (the same
// deterministic steps, so the same results); the update's buckets (gather form) or found
// entries (scatter form, with the int64 sums of all ranks added through distributed shared
// memory) and the candidates' location and estimation are split into contiguous shares; rank
// 0 gathers the candidates' results and merges.  Each item is computed exactly as by one CTA,
// so the outputs do not depend on csize.
template <int RMAX>
__device__ __forceinline__ void decode_body(const DecodeArgs& a, const int sig, const int crank = 0,
                                            const int csize = 1) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ uint32_t s_par[3];
    __shared__ int s_ws[33];
    __shared__ int s_hist[512];
    __shared__ int s_bc[4];
    __shared__ int s_cnt;
    __shared__ unsigned s_max;
    __shared__ float s_theta;
    __shared__ int s_fx;
    // the iteration's tables the location reads level by level (a chain of dependent loads per
    // candidate), copied to shared memory: offsets, vote thresholds and phase scales here, the
    // block centres and region shifts (l per block level) after the update, past the bucket
    // arrays of the selection and location (decode_smem leaves room for them)
    __shared__ uint32_t s_tau[RMAX];
    __shared__ uint32_t s_H[RMAX];
    __shared__ float s_jscale[RMAX];
    const IterDev* __restrict__ it = a.it;
    const int tid = threadIdx.x, T = blockDim.x;
    const int B = it->B, R = it->R, S = it->S, logL = it->logL;
    const uint32_t L = (uint32_t)it->L;
    const uint32_t N = (uint32_t)a.N, mask = N - 1, halfN = N >> 1;
    const int n = a.n, shift = 32 - n;
    float2* Y = a.y + (int64_t)sig * a.y_stride;
    int32_t* ff = a.ff + (int64_t)sig * a.Fcap;
    double2* fv = a.fv + (int64_t)sig * a.Fcap;
    int8_t* fvotes = a.fvotes + (int64_t)sig * a.Fcap;
    int32_t* hk = a.hkeys + ((int64_t)sig << a.Hlog);
    int32_t* hv = a.hvals + ((int64_t)sig << a.Hlog);
    for (int i = tid; i < R; i += T) {
        s_tau[i] = (uint32_t)it->tau[i];
        if (i < S) {
            s_H[i] = it->H[i];
            s_jscale[i] = it->jscale[i];
        }
    }
    if (tid == 0) {
        uint64_t s, o;
        permutation_draw(a.seed, (uint64_t)(a.signal0 + sig), (uint64_t)it->m, a.N, &s, &o);
        s_par[0] = (uint32_t)s;
        s_par[1] = (uint32_t)o;
        s_par[2] = (uint32_t)inv_odd64(s) & (uint32_t)(a.N - 1);
        s_cnt = 0;
        s_max = 0;
        s_fx = a.first ? 0 : a.fxexp[sig];
    }
    __syncthreads();
    const uint32_t sigma = s_par[0], aoff = s_par[1], sinv = s_par[2];
    const int F0 = a.F[sig];

    // shared memory (bytes, 26 B in total): [0, 16B) the update's int64 accumulators, later
    // reused for candidate results (frequency [0,4B), value [4B,12B), votes [12B,13B));
    // keys [16B,20B); candidate list [20B,22B); found-set lookups [22B,26B)
    long long* acc = (long long*)smraw;
    int32_t* cf = (int32_t*)smraw;
    float2* cv = (float2*)(smraw + 4 * (size_t)B);
    int8_t* cvt = (int8_t*)(smraw + 12 * (size_t)B);
    float* key = (float*)(smraw + 16 * (size_t)B);
    uint16_t* cand = (uint16_t*)(smraw + 20 * (size_t)B);
    int32_t* cexist = (int32_t*)(smraw + 22 * (size_t)B);

    // ---- 1. update: yhat' = yhat - yhat_update (Section 3.1, iteration steps 2-3) ------
    // Each found (f, v) adds G'^_{b'L-u} v e^{2 pi i f o_r / N} to buckets b' = b(u)-1..b(u)+1
    // of every round r.  Contributions accumulate in int64 fixed point (2^(fx-40) units,
    // fx = exponent of the largest bucket of iteration 1), so the sum does not depend on the
    // order of the additions.  Gather form: the found entries (v, f and G'^ for their three
    // buckets) are staged in shared memory in bucket order, stably (found-set order within a
    // bucket); per pass of kUpdRounds rounds the rotated values v e^{2 pi i f o_r / N} are
    // computed once per entry, then each (bucket b', split) work item sums the entries of
    // b'-1, b', b'+1 in FP32 in that fixed order and converts the sum once; with several
    // splits per bucket (B < block size) the items' int64 sums are added in a fixed order.  For
    // B > kGatherMaxB, or when the staged entries do not fit in shared memory, the entries
    // scatter their contributions with integer atomics into warp-private accumulator copies
    // instead (the same integer sums).
    if (!a.first && F0 > 0) {
        const int fx = s_fx;
        const float scale = ldexpf(1.f, 40 - fx);
        const float iscale = ldexpf(1.f, fx - 40);
        // shared memory: bucket offsets, then per staged entry v (float2), f, G'^ (3), and the
        // rotated values c_r = v e^{2 pi i f o_r / N} of the current pass (kUpdRounds float2),
        // then (several splits per bucket) the splits' partial sums
        const size_t off_v = ((size_t)4 * (2 * B + 1) + 7) & ~(size_t)7;
        const size_t off_c = off_v + (size_t)8 * F0;
        const size_t off_f = off_c + (size_t)8 * kUpdRounds * F0;
        const size_t off_g = off_f + (size_t)4 * F0;
        const size_t acc_off = (off_g + (size_t)12 * F0 + 15) & ~(size_t)15;
        // splits per bucket: enough items for every thread when B < T, as many as the
        // partial sums leave room for
        int splits = B < T ? T / B : 1;
        while (splits > 1 && acc_off + (size_t)16 * kUpdRounds * splits * B > decode_smem(B)) splits >>= 1;
        const size_t need = acc_off + (splits > 1 ? (size_t)16 * kUpdRounds * splits * B : 0);
        if (B <= kGatherMaxB && need <= decode_smem(B)) {
            int* cnt = (int*)smraw;          // B + 1: counts, then offsets of each bucket's entries
            int* fillp = cnt + (B + 1);      // B: placement cursors
            float2* ev = (float2*)(smraw + off_v);
            float2* ec = (float2*)(smraw + off_c);
            uint32_t* ef = (uint32_t*)(smraw + off_f);
            float* eg = (float*)(smraw + off_g);
            long long* part = (long long*)(smraw + acc_off);
            for (int b = tid; b <= B; b += T) cnt[b] = 0;
            __syncthreads();
            int* tb = (int*)(smraw + off_c);  // each entry's bucket (area of the rotated values)
            for (int e = tid; e < F0; e += T) {
                const uint32_t u = (sigma * (uint32_t)ff[e]) & mask;
                const int b0 = (int)(((u + (L >> 1)) >> logL) & (uint32_t)(B - 1));
                tb[e] = b0;
                atomicAdd(&cnt[b0], 1);
            }
            __syncthreads();
            {
                const int Eb = (B + T - 1) / T;
                const int lo = min(B, tid * Eb), hi = min(B, lo + Eb);
                int loc = 0;
                for (int b = lo; b < hi; ++b) loc += cnt[b];
                int tot;
                int run = block_exscan(loc, s_ws, &tot);
                for (int b = lo; b < hi; ++b) {
                    const int c = cnt[b];
                    cnt[b] = run;
                    fillp[b] = run;
                    run += c;
                }
                if (tid == 0) cnt[B] = tot;
            }
            __syncthreads();
            // stable placement: within a bucket, entries keep their found-set order, so that each
            // item below adds its entries in a fixed order.  Warp w takes a contiguous share of
            // the entries and counts them per bucket (ranks among equal buckets from warp
            // matches); an exclusive scan over the warps of each bucket then gives every entry
            // its place.  The per-warp counts go past the staged entries, each entry's bucket and
            // rank in its warp's share into the area of the rotated values (unused until the
            // passes below).
            const int lane = tid & 31, wid = tid >> 5, nw = (T + 31) >> 5;
            int* M = (int*)(smraw + acc_off);  // [nw][B]
            if (acc_off + (size_t)4 * nw * B <= decode_smem(B)) {
                int* tr = tb + F0;
                const int chunk = ((F0 + nw - 1) / nw + 31) & ~31;
                for (int i = tid; i < nw * B; i += T) M[i] = 0;
                __syncthreads();
                const int e0 = min(F0, wid * chunk), e1 = min(F0, e0 + chunk);
                int* Mw = M + wid * B;
                for (int c0 = e0; c0 < e1; c0 += 32) {
                    const int e = c0 + lane;
                    const bool has = e < e1;
                    const int b0 = has ? tb[e] : B + lane;  // a key of its own without an entry
                    const unsigned grp = __match_any_sync(0xffffffffu, b0);
                    const int rank = __popc(grp & ((1u << lane) - 1u));
                    if (has) tr[e] = Mw[b0] + rank;
                    __syncwarp();
                    if (has && rank == 0) Mw[b0] += __popc(grp);
                    __syncwarp();
                }
                __syncthreads();
                for (int bb = tid; bb < B; bb += T) {
                    int run = cnt[bb];
                    for (int w = 0; w < nw; ++w) {
                        const int t = M[w * B + bb];
                        M[w * B + bb] = run;
                        run += t;
                    }
                }
                __syncthreads();
                for (int e = tid; e < F0; e += T) {
                    const uint32_t f = (uint32_t)ff[e];
                    const double2 vd = fv[e];
                    const uint32_t u = (sigma * f) & mask;
                    const int b0 = tb[e];
                    const int pos = M[(e / chunk) * B + b0] + tr[e];
                    ev[pos] = make_float2((float)vd.x, (float)vd.y);
                    ef[pos] = f;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const int bb = (b0 + q - 1) & (B - 1);
                        const int k = (int)((((uint32_t)bb * L - u) + halfN) & mask) - (int)halfN;
                        eg[3 * pos + q] = it->Ghat[k < 0 ? -k : k] * scale;
                    }
                }
                __syncthreads();
            } else {
                // the warps of a chunk take their turn in order
                for (int c0 = 0; c0 < F0; c0 += T) {
                    const int e = c0 + tid;
                    const bool has = e < F0;
                    uint32_t f = 0;
                    float2 ve = make_float2(0.f, 0.f);
                    int b0 = B + lane;  // a key of its own for lanes without an entry
                    float g3[3] = {0.f, 0.f, 0.f};
                    if (has) {
                        f = (uint32_t)ff[e];
                        const double2 vd = fv[e];
                        ve = make_float2((float)vd.x, (float)vd.y);
                        const uint32_t u = (sigma * f) & mask;
                        b0 = (int)(((u + (L >> 1)) >> logL) & (uint32_t)(B - 1));
    #pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const int bb = (b0 + q - 1) & (B - 1);
                            const int k = (int)((((uint32_t)bb * L - u) + halfN) & mask) - (int)halfN;
                            g3[q] = it->Ghat[k < 0 ? -k : k] * scale;
                        }
                    }
                    const unsigned grp = __match_any_sync(0xffffffffu, b0);
                    const int rank = __popc(grp & ((1u << lane) - 1u));
                    for (int w = 0; w < nw; ++w) {
                        if (wid == w) {
                            if (has) {
                                const int pos = fillp[b0] + rank;
                                ev[pos] = ve;
                                ef[pos] = f;
    #pragma unroll
                                for (int q = 0; q < 3; ++q) eg[3 * pos + q] = g3[q];
                            }
                            __syncwarp();
                            if (has && rank == 0) fillp[b0] += __popc(grp);
                        }
                        __syncthreads();
                    }
                }
            }
            int b_lo, b_hi;
            rank_share(B, crank, csize, &b_lo, &b_hi);
            const int Bc = b_hi - b_lo;
            for (int r0 = 0; r0 < R; r0 += kUpdRounds) {
                const int nr = min(kUpdRounds, R - r0);
                // round-major (ec[rr F0 + j]): the entries a warp gathers below fall in
                // different banks (entry-major rows of 32 bytes would share 4 bank positions)
                for (int pos = tid; pos < F0; pos += T) {
                    const float2 v = ev[pos];
                    const uint32_t f = ef[pos];
#pragma unroll
                    for (int rr = 0; rr < kUpdRounds; ++rr) {
                        if (rr < nr) {
                            const uint32_t o_r = (aoff + sigma * s_tau[r0 + rr]) & mask;
                            ec[rr * F0 + pos] = cmul(v, cis_2pi_frac((f * o_r) & mask, n));
                        }
                    }
                }
                __syncthreads();
                for (int item = tid; item < Bc * splits; item += T) {
                    const int bp = b_lo + item % Bc, sp = item / Bc;
                    // the item's few entries add in FP32 in their staged (fixed) order; the
                    // items' sums then add exactly in int64
                    float fr[kUpdRounds], fi[kUpdRounds];
#pragma unroll
                    for (int rr = 0; rr < kUpdRounds; ++rr) fr[rr] = fi[rr] = 0.f;
#pragma unroll
                    for (int q = -1; q <= 1; ++q) {
                        // entries of bucket bp + q reach bp with their G'^ at offset -q
                        const int bb = (bp + q) & (B - 1);
                        const int j1 = cnt[bb + 1];
                        for (int j = cnt[bb] + sp; j < j1; j += splits) {
                            const float g = eg[3 * j + 1 - q];
#pragma unroll
                            for (int rr = 0; rr < kUpdRounds; ++rr) {
                                if (rr < nr) {
                                    const float2 c = ec[rr * F0 + j];
                                    fr[rr] = fmaf(g, c.x, fr[rr]);
                                    fi[rr] = fmaf(g, c.y, fi[rr]);
                                }
                            }
                        }
                    }
                    long long ar[kUpdRounds], ai[kUpdRounds];
#pragma unroll
                    for (int rr = 0; rr < kUpdRounds; ++rr) {
                        ar[rr] = f2ll_rn(fr[rr]);
                        ai[rr] = f2ll_rn(fi[rr]);
                    }
                    if (splits == 1) {
#pragma unroll
                        for (int rr = 0; rr < kUpdRounds; ++rr) {
                            if (rr < nr) {
                                float2* yp = &Y[(int64_t)(r0 + rr) * B + bp];
                                float2 yv = *yp;
                                yv.x -= ll2f_rn(ar[rr]) * iscale;
                                yv.y -= ll2f_rn(ai[rr]) * iscale;
                                *yp = yv;
                            }
                        }
                    } else {
#pragma unroll
                        for (int rr = 0; rr < kUpdRounds; ++rr) {
                            long long* pp = part + 2 * ((size_t)(sp * kUpdRounds + rr) * B + bp);
                            pp[0] = ar[rr];
                            pp[1] = ai[rr];
                        }
                    }
                }
                if (splits > 1) {
                    __syncthreads();
                    for (int e = tid; e < nr * Bc; e += T) {
                        const int rr = e / Bc, b = b_lo + e - rr * Bc;
                        long long sr = 0, si = 0;
                        for (int sp = 0; sp < splits; ++sp) {
                            const long long* pp = part + 2 * ((size_t)(sp * kUpdRounds + rr) * B + b);
                            sr += pp[0];
                            si += pp[1];
                        }
                        float2* yp = &Y[(int64_t)(r0 + rr) * B + b];
                        float2 yv = *yp;
                        yv.x -= ll2f_rn(sr) * iscale;
                        yv.y -= ll2f_rn(si) * iscale;
                        *yp = yv;
                    }
                }
                __syncthreads();
            }
        } else {
            const size_t budget = decode_smem(B) / sizeof(long long);  // int64 slots available
            const int per_round = 2 * B;
            int rc = (int)((size_t)R < budget / per_round ? (size_t)R : budget / per_round);
            if (rc < 1) rc = 1;
            const size_t ncmax = budget / ((size_t)rc * per_round);
            int nco = (int)((size_t)(T >> 5) < ncmax ? (size_t)(T >> 5) : ncmax);
            if (nco < 1) nco = 1;
            long long* wacc = acc + (size_t)((tid >> 5) % nco) * rc * per_round;
            int e_lo, e_hi, b_lo, b_hi;
            rank_share(F0, crank, csize, &e_lo, &e_hi);
            rank_share(B, crank, csize, &b_lo, &b_hi);
            const int Bc = b_hi - b_lo;
            for (int r0 = 0; r0 < R; r0 += rc) {
                const int nr = min(rc, R - r0);
                for (int i = tid; i < nco * rc * per_round; i += T) acc[i] = 0;
                __syncthreads();
                for (int i = e_lo + tid; i < e_hi; i += T) {
                    const uint32_t f = (uint32_t)ff[i];
                    const double2 vd = fv[i];
                    const float2 v = make_float2((float)vd.x, (float)vd.y);
                    const uint32_t u = (sigma * f) & mask;
                    const int b0 = (int)(((u + (L >> 1)) >> logL) & (uint32_t)(B - 1));
                    float g3[3];
                    int bb[3];
    #pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        bb[q] = (b0 + q - 1) & (B - 1);
                        const int k = (int)((((uint32_t)bb[q] * L - u) + halfN) & mask) - (int)halfN;
                        g3[q] = it->Ghat[k < 0 ? -k : k] * scale;
                    }
                    for (int rr = 0; rr < nr; ++rr) {
                        const uint32_t o_r = (aoff + sigma * s_tau[r0 + rr]) & mask;
                        const float2 c = cmul(v, cis_2pi_frac((f * o_r) & mask, n));
                        long long* ar = wacc + (size_t)rr * per_round;
    #pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            atomicAdd((unsigned long long*)&ar[2 * bb[q]], (unsigned long long)f2ll_rn(g3[q] * c.x));
                            atomicAdd((unsigned long long*)&ar[2 * bb[q] + 1], (unsigned long long)f2ll_rn(g3[q] * c.y));
                        }
                    }
                }
                decode_sync(csize);  // every rank's copies are complete
                for (int e = tid; e < nr * Bc; e += T) {
                    const int rr = e / Bc, b = b_lo + e - rr * Bc;
                    long long sr = 0, si = 0;
                    for (int q = 0; q < csize; ++q) {
                        // the copies of rank q (this block's own when csize == 1)
                        const long long* aq = csize > 1 ? cg::this_cluster().map_shared_rank(acc, q) : acc;
                        for (int w = 0; w < nco; ++w) {
                            const long long* aw = aq + ((size_t)w * rc + rr) * per_round;
                            sr += aw[2 * b];
                            si += aw[2 * b + 1];
                        }
                    }
                    float2* yp = &Y[(int64_t)(r0 + rr) * B + b];
                    float2 yv = *yp;
                    yv.x -= ll2f_rn(sr) * iscale;
                    yv.y -= ll2f_rn(si) * iscale;
                    *yp = yv;
                }
                decode_sync(csize);  // no rank clears its copies while another still reads them
            }
        }
    }

    // ---- 2. large-bucket selection (Section 3: buckets with p >= 1) -------------------
    // (a cluster's ranks updated disjoint buckets: all of them are visible after this barrier;
    // the bucket rows are read past L1 from here on)
    if (csize > 1) decode_sync(csize);
    const int lb = a.l;
    uint32_t* s_Cj = (uint32_t*)(smraw + decode_tables_off(B));  // [S - 1][l]
    int32_t* s_Dj = (int32_t*)(s_Cj + (S - 1) * lb);              // [S - 1][l]
    for (int i = tid; i < (S - 1) * lb; i += T) {
        const int lv = i / lb, j = i - lv * lb;
        s_Cj[i] = it->Cj[lv][j];
        s_Dj[i] = it->Dj[lv][j];
    }
    float mx = 0.f;
    for (int b = tid; b < B; b += T) {
        const float2 y0 = __ldcg(Y + b);
        const float k2 = fmaf(y0.x, y0.x, y0.y * y0.y);
        key[b] = k2;
        mx = fmaxf(mx, k2);
    }
    if (a.first) {
        const unsigned wm = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
        if ((tid & 31) == 0) atomicMax(&s_max, wm);
        __syncthreads();
        if (tid == 0) {
            const float m = __uint_as_float(s_max);
            const float th = a.sig_floor > 0.f ? a.sig_floor * m : -1.f;
            int e = 0;
            frexpf(sqrtf(m), &e);
            if (crank == 0) {
                a.theta[sig] = th;
                a.fxexp[sig] = e;
            }
            s_theta = th;
        }
    } else if (tid == 0) {
        s_theta = a.theta[sig];
    }
    __syncthreads();
    const float theta = s_theta;
    const int n_c = it->n_c;
    int ncand;
    if (B <= 32) {
        // one warp: the rank of each key (larger first, ties to the lower bucket) decides the
        // same n_c buckets as the block-wide radix select below
        if (tid < 32) {
            const int b = tid;
            const bool valid = b < B;
            const uint32_t kb = valid ? __float_as_uint(key[b]) : 0u;
            int rank = 0;
            for (int j = 0; j < 32; ++j) {
                const uint32_t kj = __shfl_sync(0xffffffffu, kb, j);
                rank += (j < B) && (kj > kb || (kj == kb && j < b));
            }
            const bool sel = valid && (n_c >= B || rank < n_c) && key[b] > theta;
            const unsigned m = __ballot_sync(0xffffffffu, sel);
            if (sel) cand[__popc(m & ((1u << b) - 1u))] = (uint16_t)b;
            if (tid == 0) s_bc[0] = __popc(m);
        }
        __syncthreads();
        ncand = s_bc[0];
        __syncthreads();
    } else {
        // each thread owns a contiguous chunk of buckets for order-preserving scans
        const int E = (B + T - 1) / T;
        const int b_lo = min(B, tid * E), b_hi = min(B, b_lo + E);
        uint32_t Tb = 0;
        int need_ties = 0;
        if (n_c < B) {
            // T = the n_c-th largest key (keys >= 0 compare as unsigned integers)
            Tb = block_radix_select(key, b_lo, b_hi, E, n_c, s_hist, s_bc);
            int gt = 0;
            for (int b = b_lo; b < b_hi; ++b) gt += (__float_as_uint(key[b]) > Tb);
            need_ties = n_c - block_count(gt, &s_cnt);
        }
        // selection flags of this thread's chunk (E <= 4 buckets), ties to the lower b
        int ties = 0;
        for (int b = b_lo; b < b_hi; ++b) ties += (n_c < B && __float_as_uint(key[b]) == Tb);
        int tot_ties;
        int tie_rank = block_exscan(ties, s_ws, &tot_ties);
        uint32_t selmask = 0;
        int nsel_local = 0;
        for (int b = b_lo; b < b_hi; ++b) {
            const uint32_t kb = __float_as_uint(key[b]);
            bool sel;
            if (n_c >= B) sel = true;
            else if (kb > Tb) sel = true;
            else if (kb == Tb) { sel = tie_rank < need_ties; ++tie_rank; }
            else sel = false;
            sel = sel && (key[b] > theta);
            if (sel) selmask |= 1u << (b - b_lo);
            nsel_local += sel;
        }
        int pos = block_exscan(nsel_local, s_ws, &ncand);
        for (int b = b_lo; b < b_hi; ++b)
            if ((selmask >> (b - b_lo)) & 1u) cand[pos++] = (uint16_t)b;
        __syncthreads();
    }

    // ---- 3. multiscale location, votes, estimation: one thread per candidate ----------
    const int l = a.l;
    const int need = a.min_votes > 0 ? min(a.min_votes, S) : S;
    int r_lo, r_hi;  // this rank's share of the candidates
    rank_share(ncand, crank, csize, &r_lo, &r_hi);
    for (int ci = r_lo + tid; ci < r_hi; ci += T) {
        const int b = cand[ci];
        const float2 y0 = __ldcg(Y + b);
        const float m0 = fmaf(y0.x, y0.x, y0.y * y0.y);
        // phases phi_s (2^-32 turns) and magnitude votes of all levels, loaded up front
        uint32_t ph[RMAX];
        uint64_t magok = 0;
#pragma unroll
        for (int s = 1; s < RMAX; ++s) {
            if (s <= S) {
                const float2 ys = __ldcg(Y + (int64_t)s * B + b);
                ph[s - 1] = phase_fixed(ys, y0);
                const float ms = fmaf(ys.x, ys.x, ys.y * ys.y);
                magok |= (fabsf(ms - m0) <= a.mag_tol * m0) ? (1ull << (s - 1)) : 0ull;
            }
        }
        // block levels: region [u_min, u_min + Lbar_s) of l blocks
        int32_t umin = b * (int32_t)L - (int32_t)L;
#pragma unroll
        for (int s = 1; s < RMAX; ++s) {
            if (s < S) {
                const uint32_t ts = s_tau[s];
                const uint32_t Ap = ((uint32_t)umin * ts) << shift;
                const int j0 = (int)floorf((float)(ph[s - 1] - Ap) * s_jscale[s - 1]);
                uint32_t bd = 0xffffffffu;
                int bj = l;
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    const int j = q < 5 ? j0 - 2 + q : (q == 5 ? 0 : l - 1);
                    if (j < 0 || j >= l) continue;
                    const uint32_t d = circ_dist(ph[s - 1], Ap + s_Cj[(s - 1) * lb + j]);
                    if (d < bd || (d == bd && j < bj)) { bd = d; bj = j; }
                }
                umin += s_Dj[(s - 1) * lb + bj];
            }
        }
        // final level: the Lbar_S integers u_min + i
        uint32_t phS = 0;
#pragma unroll
        for (int s = 1; s < RMAX; ++s)
            if (s == S) phS = ph[s - 1];
        if (a.fine_phase) {
            // phase step 1/N: FP32 atan2 is too coarse past N ~ 2^20
            phS = phase_fixed64(__ldcg(Y + (int64_t)S * B + b), y0);
#pragma unroll
            for (int s = 1; s < RMAX; ++s)
                if (s == S) ph[s - 1] = phS;
        }
        uint32_t ustar;
        {
            const uint32_t ts = s_tau[S];
            const int Lb = (int)it->Lbar[S - 1];
            const uint32_t Dl = (uint32_t)it->W[S - 1];
            const uint32_t P0 = ((uint32_t)umin * ts) << shift;
            const int i0 = (int)floorf((float)(phS - P0) * s_jscale[S - 1]);
            uint32_t bd = 0xffffffffu;
            int bi = Lb;
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const int i = q < 5 ? i0 - 2 + q : (q == 5 ? 0 : Lb - 1);
                if (i < 0 || i >= Lb) continue;
                const uint32_t d = circ_dist(phS, P0 + (uint32_t)i * Dl);
                if (d < bd || (d == bd && i < bi)) { bd = d; bi = i; }
            }
            ustar = (uint32_t)(umin + bi) & mask;
        }
        // votes: phase consistency with u* and magnitude consistency with round 0
        int nv = 0;
#pragma unroll
        for (int s = 1; s < RMAX; ++s) {
            if (s <= S) {
                const uint32_t Ps = (ustar * s_tau[s]) << shift;
                nv += (circ_dist(ph[s - 1], Ps) <= s_H[s - 1]) && ((magok >> (s - 1)) & 1ull);
            }
        }
        const bool own = (int)(((ustar + (L >> 1)) >> logL) & (uint32_t)(B - 1)) == b;
        const bool accept = nv >= need && own;
        cvt[ci] = accept ? (int8_t)nv : (int8_t)-1;
        if (accept) {
            const uint32_t f = (sinv * ustar) & mask;
            const int kb = (int)((((uint32_t)b * L - ustar) + halfN) & mask) - (int)halfN;
            const float ig = 1.f / it->Ghat[kb < 0 ? -kb : kb];
            float vre[RMAX], vim[RMAX];
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
                if (r < R) {
                    const uint32_t o_r = (aoff + sigma * s_tau[r]) & mask;
                    const float2 e = cis_2pi_frac((f * o_r) & mask, n);
                    const float2 v = cmul(__ldcg(Y + (int64_t)r * B + b), make_float2(e.x, -e.y));
                    vre[r] = v.x * ig;
                    vim[r] = v.y * ig;
                }
            }
            cf[ci] = (int32_t)f;
            const float mre = median_of<RMAX>(vre, R);
            const float mim = median_of<RMAX>(vim, R);
            cv[ci] = make_float2(mre, mim);
        }
    }
    __syncthreads();
    if (csize > 1) {
        // the other ranks store their shares of the candidate results (cf, cv, cvt) into rank
        // 0's arrays (those indices are rank 0's only after the update, which every rank has
        // finished: the selection began with a cluster barrier)
        if (crank != 0) {
            int32_t* rf = cg::this_cluster().map_shared_rank(cf, 0);
            float2* rv = cg::this_cluster().map_shared_rank(cv, 0);
            int8_t* rt = cg::this_cluster().map_shared_rank(cvt, 0);
            for (int ci = r_lo + tid; ci < r_hi; ci += T) {
                rt[ci] = cvt[ci];
                if (cvt[ci] >= 0) {
                    rf[ci] = cf[ci];
                    rv[ci] = cv[ci];
                }
            }
        }
        decode_sync(csize);  // rank 0 holds every candidate's result
        if (crank != 0) return;
    }

    // ---- 4. merge: x^m = x^{m-1} + x'^m (Section 3.1, step 5) -------------------------
    for (int ci = tid; ci < ncand; ci += T)
        cexist[ci] = (cvt[ci] >= 0) ? hash_find(hk, hv, a.Hlog, cf[ci]) : -2;
    __syncthreads();
    const int cE = (ncand + T - 1) / T;
    const int c_lo = min(ncand, tid * cE), c_hi = min(ncand, c_lo + cE);
    int nnew_local = 0;
    for (int ci = c_lo; ci < c_hi; ++ci) nnew_local += (cexist[ci] == -1);
    int nnew;
    int npos = block_exscan(nnew_local, s_ws, &nnew);
    for (int ci = c_lo; ci < c_hi; ++ci) {
        const int ex = cexist[ci];
        if (ex >= 0) {
            double2 v = fv[ex];
            v.x += (double)cv[ci].x;
            v.y += (double)cv[ci].y;
            fv[ex] = v;
        } else if (ex == -1) {
            const int e = F0 + npos++;
            ff[e] = cf[ci];
            fv[e] = make_double2((double)cv[ci].x, (double)cv[ci].y);
            fvotes[e] = cvt[ci];
            hash_insert(hk, hv, a.Hlog, cf[ci], e);
        }
    }
    if (tid == 0) a.F[sig] = F0 + nnew;
}

template <int RMAX>
__global__ void __launch_bounds__(kDecodeThreads, 2) k_decode(const DecodeArgs a) {
    decode_body<RMAX>(a, blockIdx.x);
}

// The decode of each signal spread over a thread-block cluster (launched with a cluster
// dimension of csize along x; cluster c decodes signal c): the one-signal latency path.
template <int RMAX>
__global__ void __launch_bounds__(kDecodeThreads, 2) k_decode_cluster(const DecodeArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const int csize = (int)cl.num_blocks();
    decode_body<RMAX>(a, blockIdx.x / csize, (int)cl.block_rank(), csize);
}

// Batch of signals with different N and K: CTA b decodes signal jobs[list[b]], whose
// DecodeArgs already point at that signal's own workspace (so it is signal 0 of its args).
template <int RMAX>
__global__ void __launch_bounds__(kDecodeThreads, 2) k_decode_multi(const DecodeArgs* __restrict__ jobs,
                                                                 const int32_t* __restrict__ list) {
    __shared__ __align__(16) DecodeArgs sa;
    const DecodeArgs* src = jobs + list[blockIdx.x];
    for (int i = threadIdx.x; i < (int)(sizeof(DecodeArgs) / 4); i += blockDim.x)
        ((uint32_t*)&sa)[i] = ((const uint32_t*)src)[i];
    __syncthreads();
    decode_body<RMAX>(sa, 0);
}

// Persistent decode of a batch of signals of different sizes: each CTA takes whole signals
// from a device queue (the next unclaimed entry of `order`, longest decode chains first) and
// runs that signal's iterations in order, jobs[off[i]] .. jobs[off[i] + len[i] - 1], each
// exactly as k_decode_multi runs it.  No CTA waits for another: a signal's iterations depend
// only on each other, and all its bucket arrays exist before the launch.  *queue must be 0 at
// launch.
template <int RMAX>
__global__ void __launch_bounds__(kDecodeThreads, 2) k_decode_chain(const DecodeArgs* __restrict__ jobs,
                                                                 const int32_t* __restrict__ off,
                                                                 const int32_t* __restrict__ len,
                                                                 const int32_t* __restrict__ order, int nsig,
                                                                 int32_t* queue) {
    __shared__ __align__(16) DecodeArgs sa;
    __shared__ int s_q;
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(queue, 1);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        if (q >= nsig) break;
        const int i = order[q];
        for (int k = 0; k < len[i]; ++k) {
            const DecodeArgs* src = jobs + off[i] + k;
            for (int w = threadIdx.x; w < (int)(sizeof(DecodeArgs) / 4); w += blockDim.x)
                ((uint32_t*)&sa)[w] = ((const uint32_t*)src)[w];
            __syncthreads();
            decode_body<RMAX>(sa, 0);
            __syncthreads();
        }
    }
}

// Persistent decode of a uniform batch: each CTA takes signals from a device queue and runs
// iterations 1..M of that signal in order, iteration m exactly as k_decode runs it for the
// signal.  All bucket arrays exist before the launch; no CTA waits for another.  *queue must be
// 0 at launch.
template <int RMAX>
__global__ void __launch_bounds__(kDecodeThreads, 2) k_decode_chain_uniform(const DecodeArgs* __restrict__ iters,
                                                                         int M, int nsig, int32_t* queue) {
    __shared__ __align__(16) DecodeArgs sa;
    __shared__ int s_q;
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(queue, 1);
        __syncthreads();
        const int sig = s_q;
        __syncthreads();
        if (sig >= nsig) break;
        for (int mi = 0; mi < M; ++mi) {
            for (int w = threadIdx.x; w < (int)(sizeof(DecodeArgs) / 4); w += blockDim.x)
                ((uint32_t*)&sa)[w] = ((const uint32_t*)(iters + mi))[w];
            __syncthreads();
            decode_body<RMAX>(sa, sig);
            __syncthreads();
        }
    }
}

// ----------------------------------------------------------------- finalize ---------
// Top-K of the found set by |v| (ties to the lower frequency), sorted by frequency.
__device__ __forceinline__ void finalize_body(const int32_t* Fc, const int32_t* ffa,
                                              const double2* fva, const int8_t* fvta,
                                              int64_t Fcap, int64_t K, int64_t Kout,
                                              int64_t* idx_out, sfft4_c128* val_out,
                                              int64_t* nfound_out, int8_t* votes_out,
                                              const int sig, const int osig) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long* srt = (unsigned long long*)smraw;  // (f << 32 | entry), pow2 >= K
    __shared__ int s_cnt;
    __shared__ int s_ws[33];
    const int tid = threadIdx.x, T = blockDim.x;
    const int F0 = Fc[sig];
    const int32_t* ff = ffa + (int64_t)sig * Fcap;
    const double2* fv = fva + (int64_t)sig * Fcap;
    const int8_t* fvt = fvta + (int64_t)sig * Fcap;
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    auto keyof = [&](int i) -> unsigned long long {
        const double2 v = fv[i];
        return (unsigned long long)__double_as_longlong(v.x * v.x + v.y * v.y);
    };
    unsigned long long Tk = 0;
    int32_t fT = 0x7fffffff;
    const bool cut = F0 > K;
    if (cut) {
        for (int bit = 62; bit >= 0; --bit) {
            const unsigned long long trial = Tk | (1ull << bit);
            int c = 0;
            for (int i = tid; i < F0; i += T) c += keyof(i) >= trial;
            if (block_count(c, &s_cnt) >= K) Tk = trial;
        }
        int gt = 0;
        for (int i = tid; i < F0; i += T) gt += keyof(i) > Tk;
        const int need = (int)K - block_count(gt, &s_cnt);
        // among ties at Tk keep the `need` lowest frequencies
        int32_t lo = 0;
        for (int bit = 30; bit >= 0; --bit) {
            const int32_t trial = lo | (1 << bit);
            int c = 0;
            for (int i = tid; i < F0; i += T) c += (keyof(i) == Tk) && (ff[i] < trial);
            if (block_count(c, &s_cnt) < need) lo = trial;
        }
        fT = lo;  // ties with f <= fT are kept
    }
    const int E = (F0 + T - 1) / T;
    const int e_lo = min(F0, tid * E), e_hi = min(F0, e_lo + E);
    int nl = 0;
    for (int i = e_lo; i < e_hi; ++i) {
        const unsigned long long k = keyof(i);
        nl += !cut || k > Tk || (k == Tk && ff[i] <= fT);
    }
    int nsel;
    int pos = block_exscan(nl, s_ws, &nsel);
    int P2 = 1;
    while (P2 < nsel) P2 <<= 1;
    for (int i = tid; i < P2; i += T) srt[i] = ~0ull;
    __syncthreads();
    for (int i = e_lo; i < e_hi; ++i) {
        const unsigned long long k = keyof(i);
        if (!cut || k > Tk || (k == Tk && ff[i] <= fT))
            srt[pos++] = ((unsigned long long)(uint32_t)ff[i] << 32) | (uint32_t)i;
    }
    __syncthreads();
    for (int kk = 2; kk <= P2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P2; i += T) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a0 = srt[i], b0 = srt[ixj];
                    const bool up = (i & kk) == 0;
                    if ((a0 > b0) == up) { srt[i] = b0; srt[ixj] = a0; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < Kout; i += T) {
        const int64_t o = (int64_t)osig * Kout + i;
        if (i < nsel) {
            const int e = (int)(srt[i] & 0xffffffffu);
            idx_out[o] = (int64_t)(srt[i] >> 32);
            val_out[o].re = fv[e].x;
            val_out[o].im = fv[e].y;
            if (votes_out) votes_out[o] = fvt[e];
        } else {
            idx_out[o] = -1;
            val_out[o].re = 0;
            val_out[o].im = 0;
            if (votes_out) votes_out[o] = 0;
        }
    }
    if (tid == 0) nfound_out[osig] = nsel;
}

__global__ void __launch_bounds__(1024) k_finalize(const int32_t* Fc, const int32_t* ffa,
                                                   const double2* fva, const int8_t* fvta,
                                                   int64_t Fcap, int64_t K, int64_t* idx_out,
                                                   sfft4_c128* val_out, int64_t* nfound_out,
                                                   int8_t* votes_out) {
    finalize_body(Fc, ffa, fva, fvta, Fcap, K, K, idx_out, val_out, nfound_out, votes_out, blockIdx.x,
                  blockIdx.x);
}

// Batch of signals with different K: job b finalises signal slot b (its found set at its own
// workspace), writing row b of outputs of row length Kout (entries past the signal's K = -1).

__global__ void __launch_bounds__(1024) k_finalize_multi(const FinalJob* __restrict__ jobs, int64_t Kout,
                                                         int64_t* idx_out, sfft4_c128* val_out,
                                                         int64_t* nfound_out, int8_t* votes_out) {
    const FinalJob j = jobs[blockIdx.x];
    finalize_body(j.F, j.ff, j.fv, j.fvt, j.Fcap, j.K, Kout, idx_out, val_out, nfound_out, votes_out, 0,
                  blockIdx.x);
}

// Histogram of the votes of every found-set entry of jobs[blockIdx.x]'s signal.
__global__ void __launch_bounds__(256) k_votes_hist(const FinalJob* __restrict__ jobs,
                                                    unsigned long long* __restrict__ hist) {
    __shared__ unsigned int h[SFFT4_MAX_VOTES + 1];
    for (int i = threadIdx.x; i <= SFFT4_MAX_VOTES; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const FinalJob j = jobs[blockIdx.x];
    const int F = *j.F;
    for (int e = threadIdx.x; e < F; e += blockDim.x) {
        const int v = j.fvt[e];
        atomicAdd(&h[v < 0 ? 0 : (v > SFFT4_MAX_VOTES ? SFFT4_MAX_VOTES : v)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= SFFT4_MAX_VOTES; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// ----------------------------------------------------------------- launchers --------
int configure_kernels();

FoldArgs make_fold_args(const sfft4_plan_s* p, int mi, const FoldGroup& g, size_t* smem_out) {
    const IterHost& ih = p->iters[mi];
    const IterDev& d = ih.d;
    FoldArgs a;
    memset(&a, 0, sizeof(a));
    a.z_stride = (int64_t)p->R_max * p->B_max;
    a.N = (uint64_t)p->N;
    a.seed = p->seed;
    a.m = d.m;
    a.B = d.B;
    a.logB = d.logB;
    a.Wj = ih.Wj;
    a.h = d.h;
    a.w = 2 * d.h + 1;
    a.G = d.G;
    a.g = g;
    for (int s = 0; s < kFoldRG; ++s) a.tau[s] = (s < g.nr) ? (int32_t)d.tau[g.r0 + s] : 0;
    if (smem_out) *smem_out = fold_smem(g.nr, ih.Wj * g.P);
    return a;
}

// B-point DFT of every (signal, round) column of iteration mi: z holds signal s's R x B
// folded arrays at z + s z_stride, y receives the bucket arrays at y + s y_stride.
int launch_iter_dft(sfft4_plan_s* p, int mi, int nsig, const float2* z, int64_t z_stride, float2* y_out,
                    int64_t y_sig_stride, cudaStream_t st) {
    const IterHost& ih = p->iters[mi];
    const IterDev& d = ih.d;
    const int B = d.B, logB = d.logB, R = d.R;
    int T = std::min(1024, std::max(256, B / 2));
    int cpc = std::max(1, (2 * T) / B);
    int ncols = nsig * R;
    int blocks = (ncols + cpc - 1) / cpc;
    size_t smem = (size_t)cpc * B * sizeof(float2);
    cudaEvent_t ev = nullptr;
    int rc = prof_begin(p, st, &ev);
    if (rc) return rc;
    if (p->o.precision == SFFT4_BF16X3) {
        const Window& w = p->wins[ih.win];
        rc = launch_dft_tc(z, z_stride, p->u, (int64_t)p->R_max * p->B_max, y_out, y_sig_stride, nsig, R, B,
                           w.dA1, w.dA2, w.tw4, p->status, p->sm_count, st);
    } else {
        k_fft<<<blocks, T, smem, st>>>(z, y_out, B, logB, d.tw, z_stride, y_sig_stride, R, cpc, ncols,
                                       nullptr, nullptr);
        rc = check_cuda(cudaGetLastError());
    }
    if (rc) return rc;
    const int Bi = (int)B;
    return prof_end(p, st, ev, kProfFft, 0, p->o.precision == SFFT4_BF16X3 ? dft_tc_launches(&Bi, 1) : 1);
}

int launch_bucketize(sfft4_plan_s* p, int mi, int nsig, const float2* x, int64_t x_stride,
                     int32_t signal0, float2* y_out, int64_t y_sig_stride, cudaStream_t st) {
    int rc0 = configure_kernels();
    if (rc0) return rc0;
    const IterHost& ih = p->iters[mi];
    const IterDev& d = ih.d;
    for (const FoldGroup& g : ih.groups) {
        size_t smem = 0;
        FoldArgs a = make_fold_args(p, mi, g, &smem);
        a.x = x;
        a.x_stride = x_stride;
        a.z = p->z;
        a.signal0 = signal0;
        dim3 grid(d.B / ih.Wj, nsig);
        int threads = ih.Wj * g.P;
        cudaEvent_t ev = nullptr;
        int rc = prof_begin(p, st, &ev);
        if (rc) return rc;
        switch (g.nr) {
            case 1: k_fold<1><<<grid, threads, smem, st>>>(a); break;
            case 2: k_fold<2><<<grid, threads, smem, st>>>(a); break;
            case 3: k_fold<3><<<grid, threads, smem, st>>>(a); break;
            case 4: k_fold<4><<<grid, threads, smem, st>>>(a); break;
            case 5: k_fold<5><<<grid, threads, smem, st>>>(a); break;
            case 6: k_fold<6><<<grid, threads, smem, st>>>(a); break;
            case 7: k_fold<7><<<grid, threads, smem, st>>>(a); break;
            default: k_fold<8><<<grid, threads, smem, st>>>(a); break;
        }
        rc = prof_end(p, st, ev, kProfFold, g.unique * nsig);
        if (rc) return rc;
    }
    return launch_iter_dft(p, mi, nsig, p->z, (int64_t)p->R_max * p->B_max, y_out, y_sig_stride, st);
}

DecodeArgs make_decode_args(const sfft4_plan_s* p, int mi) {
    DecodeArgs a;
    memset(&a, 0, sizeof(a));
    a.N = (uint64_t)p->N;
    a.seed = p->seed;
    a.n = p->n;
    a.signal0 = 0;
    a.first = (mi == 0);
    a.l = p->l;
    a.qn = p->qn;
    a.min_votes = p->o.min_votes;
    a.fine_phase = p->o.location == SFFT4_LOC_TWO_ROUND;
    a.mag_tol = (float)p->o.mag_tol;
    a.sig_floor = (float)p->o.sig_floor;
    a.it = p->iters_dev + mi;
    a.y = p->y + p->yoff[mi];
    a.y_stride = p->ytot;
    a.F = p->F;
    a.ff = p->ff;
    a.fv = p->fv;
    a.fvotes = p->fvotes;
    a.Fcap = p->Fcap;
    a.hkeys = p->hkeys;
    a.hvals = p->hvals;
    a.Hlog = p->Hlog;
    a.theta = p->theta;
    a.fxexp = p->fxexp;
    return a;
}

// CTAs per signal of the decode: opts.decode_cluster, or (0) the largest power of two up to 8
// with which the batch's decode CTAs still fit on the SMs, so that a small batch spreads each
// signal's decode over several SMs instead of leaving them idle.
int decode_cluster_size(const sfft4_plan_s* p, int nsig) {
    if (p->o.decode_cluster > 0) return p->o.decode_cluster;
    // 4 measured fastest from 1 to 32 signals of N = 2^22, K = 1000 (one signal: 434 us per
    // execute against 449 us with 8; 16 signals: 574 against 636 us), 2 at 64 signals
    int c = 4;
    while (c > 1 && (int64_t)nsig * c > p->sm_count) c >>= 1;
    return c;
}

int launch_decode(sfft4_plan_s* p, int mi, int nsig, cudaStream_t st) {
    int rc0 = configure_kernels();
    if (rc0) return rc0;
    const IterDev& d = p->iters[mi].d;
    DecodeArgs a = make_decode_args(p, mi);
    size_t smem = decode_smem(d.B);
    cudaEvent_t ev = nullptr;
    int rc = prof_begin(p, st, &ev);
    if (rc) return rc;
    const int C = decode_cluster_size(p, nsig);
    if (C > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nsig * C));
        cfg.blockDim = dim3(kDecodeThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (d.R <= 8) rc = check_cuda(cudaLaunchKernelEx(&cfg, k_decode_cluster<8>, a));
        else if (d.R <= 16) rc = check_cuda(cudaLaunchKernelEx(&cfg, k_decode_cluster<16>, a));
        else rc = check_cuda(cudaLaunchKernelEx(&cfg, k_decode_cluster<64>, a));
    } else {
        if (d.R <= 8) k_decode<8><<<nsig, kDecodeThreads, smem, st>>>(a);
        else if (d.R <= 16) k_decode<16><<<nsig, kDecodeThreads, smem, st>>>(a);
        else k_decode<64><<<nsig, kDecodeThreads, smem, st>>>(a);
        rc = check_cuda(cudaGetLastError());
    }
    if (rc) return rc;
    return prof_end(p, st, ev, kProfDecode, 0);
}

size_t decode_smem_bytes(int B) { return decode_smem(B); }

// ---- launches of a batch of signals with different sizes (job tables in device memory) --
int launch_fold_multi(int RG, const FoldArgs* jobs, const FoldTile* tiles, int ntiles,
                      const float2* const* xptrs, int threads, size_t smem, cudaStream_t st) {
    switch (RG) {
        case 1: k_fold_multi<1><<<ntiles, threads, smem, st>>>(jobs, tiles, xptrs); break;
        case 2: k_fold_multi<2><<<ntiles, threads, smem, st>>>(jobs, tiles, xptrs); break;
        case 3: k_fold_multi<3><<<ntiles, threads, smem, st>>>(jobs, tiles, xptrs); break;
        case 4: k_fold_multi<4><<<ntiles, threads, smem, st>>>(jobs, tiles, xptrs); break;
        case 5: k_fold_multi<5><<<ntiles, threads, smem, st>>>(jobs, tiles, xptrs); break;
        case 6: k_fold_multi<6><<<ntiles, threads, smem, st>>>(jobs, tiles, xptrs); break;
        case 7: k_fold_multi<7><<<ntiles, threads, smem, st>>>(jobs, tiles, xptrs); break;
        default: k_fold_multi<8><<<ntiles, threads, smem, st>>>(jobs, tiles, xptrs); break;
    }
    return check_cuda(cudaGetLastError());
}

// Launch descriptors of the signal-major fold (built once per plan): one FoldArgs per
// (iteration, fold group) writing iteration m's folded arrays at zall + yoff[m], ordered by
// samples per residue slice, heaviest first, so that the last signals of a launch end
// together; at most kSigJobs jobs per launch.
int build_signal_major_fold(sfft4_plan_s* p) {
    struct Job {
        FoldArgs a;
        int32_t nsl, threads;
        size_t smem;
        int64_t per_tile, samples;
    };
    std::vector<Job> jobs;
    for (size_t mi = 0; mi < p->iters.size(); ++mi) {
        const IterHost& ih = p->iters[mi];
        const int nsl = ih.d.B / ih.Wj;
        for (const FoldGroup& g : ih.groups) {
            Job jb;
            jb.a = make_fold_args(p, (int)mi, g, &jb.smem);
            jb.a.z = p->zall + p->yoff[mi];
            jb.a.z_stride = p->ytot;
            jb.a.signal0 = 0;
            jb.nsl = nsl;
            jb.threads = ih.Wj * g.P;
            jb.per_tile = g.unique / nsl;
            jb.samples = g.unique;
            jobs.push_back(jb);
        }
    }
    std::stable_sort(jobs.begin(), jobs.end(), [](const Job& u, const Job& v) { return u.per_tile > v.per_tile; });
    p->sm_fold.clear();
    for (size_t j0 = 0; j0 < jobs.size(); j0 += kSigJobs) {
        SigFoldHost h;
        memset(&h, 0, sizeof(h));
        h.RG = 1;
        h.threads = 32;
        const size_t j1 = std::min(jobs.size(), j0 + (size_t)kSigJobs);
        for (size_t j = j0; j < j1; ++j) {
            const Job& jb = jobs[j];
            const int k = (int)(j - j0);
            h.L.jobs[k] = jb.a;
            h.L.start[k + 1] = h.L.start[k] + jb.nsl;
            h.RG = std::max(h.RG, (int32_t)jb.a.g.nr);
            h.threads = std::max(h.threads, jb.threads);
            h.smem = std::max(h.smem, jb.smem);
            h.samples += jb.samples;
        }
        h.L.njobs = (int32_t)(j1 - j0);
        h.L.ntiles = h.L.start[h.L.njobs];
        h.smem = fold_smem(h.RG, h.threads);
        if ((int64_t)h.L.ntiles * p->o.max_batch > (int64_t)INT32_MAX || h.threads > 512 ||
            h.smem > (size_t)kFoldSmemMax)
            return SFFT4_EINVAL;
        p->sm_fold.push_back(h);
    }
    return SFFT4_OK;
}

int launch_fold_signal_major(sfft4_plan_s* p, int nsig, const float2* x, int64_t x_stride, cudaStream_t st) {
    int rc0 = configure_kernels();
    if (rc0) return rc0;
    for (SigFoldHost& h : p->sm_fold) {
        h.L.x = x;
        h.L.x_stride = x_stride;
        const int grid = nsig * h.L.ntiles, th = h.threads;
        const size_t smem = h.smem;
        const SigFoldLaunch& L = h.L;
        cudaEvent_t ev = nullptr;
        int rc = prof_begin(p, st, &ev);
        if (rc) return rc;
        switch (h.RG) {
            case 1: k_fold_sig<1><<<grid, th, smem, st>>>(L); break;
            case 2: k_fold_sig<2><<<grid, th, smem, st>>>(L); break;
            case 3: k_fold_sig<3><<<grid, th, smem, st>>>(L); break;
            case 4: k_fold_sig<4><<<grid, th, smem, st>>>(L); break;
            case 5: k_fold_sig<5><<<grid, th, smem, st>>>(L); break;
            case 6: k_fold_sig<6><<<grid, th, smem, st>>>(L); break;
            case 7: k_fold_sig<7><<<grid, th, smem, st>>>(L); break;
            default: k_fold_sig<8><<<grid, th, smem, st>>>(L); break;
        }
        rc = check_cuda(cudaGetLastError());
        if (rc) return rc;
        rc = prof_end(p, st, ev, kProfFold, h.samples * nsig);
        if (rc) return rc;
    }
    return SFFT4_OK;
}

int launch_fft_multi(const float2* const* zcols, float2* const* ycols, int ncols, int B,
                     const float2* tw, cudaStream_t st) {
    int logB = 0;
    while ((1 << logB) < B) ++logB;
    int T = std::min(1024, std::max(256, B / 2));
    int cpc = std::max(1, (2 * T) / B);
    int blocks = (ncols + cpc - 1) / cpc;
    size_t smem = (size_t)cpc * B * sizeof(float2);
    k_fft<<<blocks, T, smem, st>>>(nullptr, nullptr, B, logB, tw, 0, 0, 1, cpc, ncols, zcols, ycols);
    return check_cuda(cudaGetLastError());
}

int launch_decode_multi(int rclass, const DecodeArgs* jobs, const int32_t* list, int n, size_t smem,
                        cudaStream_t st) {
    if (rclass == 0) k_decode_multi<8><<<n, kDecodeThreads, smem, st>>>(jobs, list);
    else if (rclass == 1) k_decode_multi<16><<<n, kDecodeThreads, smem, st>>>(jobs, list);
    else k_decode_multi<64><<<n, kDecodeThreads, smem, st>>>(jobs, list);
    return check_cuda(cudaGetLastError());
}

int build_decode_chain(sfft4_plan_s* p) {
    std::vector<DecodeArgs> v;
    p->dec_rclass = 0;
    p->dec_smem = 0;
    for (size_t mi = 0; mi < p->iters.size(); ++mi) {
        v.push_back(make_decode_args(p, (int)mi));
        const IterDev& d = p->iters[mi].d;
        p->dec_rclass = std::max(p->dec_rclass, d.R <= 8 ? 0 : (d.R <= 16 ? 1 : 2));
        p->dec_smem = std::max(p->dec_smem, decode_smem(d.B));
    }
    int rc = check_cuda(cudaMalloc(&p->dec_iters, v.size() * sizeof(DecodeArgs)));
    if (!rc) rc = check_cuda(cudaMemcpy(p->dec_iters, v.data(), v.size() * sizeof(DecodeArgs), cudaMemcpyHostToDevice));
    if (!rc) rc = check_cuda(cudaMalloc(&p->queue, sizeof(int32_t)));
    return rc;
}

// Synchronous executes only: in a pipeline of asynchronous executes a persistent decode would
// hold its CTA slots for the whole chain while the next batch's fold needs them (measured at
// 256 signals of N = 2^22, K = 1000: 59 K against 85 K transforms/s), whereas the decodes of
// single iterations interleave with the fold.  BF16X3 only: there every iteration's DFT runs
// in grouped launches before the first decode anyway, while the FP32 DFTs (one launch per
// iteration) overlap the decodes of earlier iterations, which the persistent decode would give
// up.  One CTA per signal only: a cluster running every iteration of one signal in one launch
// measured no faster than one launch per iteration (the gaps between launches on a stream are
// small next to the 30-40 us of each iteration's decode).
bool decode_chain_used(const sfft4_plan_s* p, int nsig) {
    return p->o.batch_exec == SFFT4_BATCH_PERSISTENT && !p->sm_fold.empty() && p->uall && !p->o.trace &&
           p->dec_iters && !p->in_async && decode_cluster_size(p, nsig) == 1;
}

int launch_decode_chain_uniform(sfft4_plan_s* p, int nsig, cudaStream_t st) {
    int rc = configure_kernels();
    if (!rc) rc = check_cuda(cudaMemsetAsync(p->queue, 0, sizeof(int32_t), st));
    if (rc) return rc;
    cudaEvent_t ev = nullptr;
    rc = prof_begin(p, st, &ev);
    if (rc) return rc;
    const int grid = std::max(1, std::min(nsig, 2 * p->sm_count));
    const int M = (int)p->iters.size();
    if (p->dec_rclass == 0) k_decode_chain_uniform<8><<<grid, kDecodeThreads, p->dec_smem, st>>>(p->dec_iters, M, nsig, p->queue);
    else if (p->dec_rclass == 1) k_decode_chain_uniform<16><<<grid, kDecodeThreads, p->dec_smem, st>>>(p->dec_iters, M, nsig, p->queue);
    else k_decode_chain_uniform<64><<<grid, kDecodeThreads, p->dec_smem, st>>>(p->dec_iters, M, nsig, p->queue);
    rc = check_cuda(cudaGetLastError());
    if (rc) return rc;
    return prof_end(p, st, ev, kProfDecode, 0);
}

int launch_decode_chain(int rclass, const DecodeArgs* jobs, const int32_t* off, const int32_t* len,
                        const int32_t* order, int nsig, int32_t* queue, int grid, size_t smem, cudaStream_t st) {
    if (rclass == 0) k_decode_chain<8><<<grid, kDecodeThreads, smem, st>>>(jobs, off, len, order, nsig, queue);
    else if (rclass == 1) k_decode_chain<16><<<grid, kDecodeThreads, smem, st>>>(jobs, off, len, order, nsig, queue);
    else k_decode_chain<64><<<grid, kDecodeThreads, smem, st>>>(jobs, off, len, order, nsig, queue);
    return check_cuda(cudaGetLastError());
}

int launch_finalize_multi(const FinalJob* jobs, int nsig, int64_t Kout, int64_t* idx, sfft4_c128* val,
                          int64_t* nfound, int8_t* votes, cudaStream_t st) {
    int P2 = 1;
    while (P2 < Kout) P2 <<= 1;
    size_t smem = (size_t)P2 * sizeof(unsigned long long);
    k_finalize_multi<<<nsig, 1024, smem, st>>>(jobs, Kout, idx, val, nfound, votes);
    return check_cuda(cudaGetLastError());
}

int launch_votes_hist(const FinalJob* jobs, int nsig, unsigned long long* hist, cudaStream_t st) {
    if (nsig < 1) return SFFT4_OK;
    k_votes_hist<<<nsig, 256, 0, st>>>(jobs, hist);
    return check_cuda(cudaGetLastError());
}

int launch_finalize(sfft4_plan_s* p, int nsig, int64_t* idx, sfft4_c128* val, int64_t* nfound,
                    int8_t* votes, cudaStream_t st) {
    int P2 = 1;
    while (P2 < p->K) P2 <<= 1;
    size_t smem = (size_t)P2 * sizeof(unsigned long long);
    cudaEvent_t ev = nullptr;
    int rc = prof_begin(p, st, &ev);
    if (rc) return rc;
    k_finalize<<<nsig, 1024, smem, st>>>(p->F, p->ff, p->fv, p->fvotes, p->Fcap, p->K, idx, val,
                                         nfound, votes);
    rc = check_cuda(cudaGetLastError());
    if (rc) return rc;
    return prof_end(p, st, ev, kProfFinalize, 0);
}

int launch_reset(sfft4_plan_s* p, int nsig, cudaStream_t st) {
    int rc = check_cuda(cudaMemsetAsync(p->F, 0, nsig * sizeof(int32_t), st));
    if (rc) return rc;
    return check_cuda(cudaMemsetAsync(p->hkeys, 0xff, ((size_t)nsig << p->Hlog) * sizeof(int32_t), st));
}

static int next_event(sfft4_plan_s* p, cudaEvent_t* e) {
    if (p->ev_used == p->ev_pool.size()) {
        cudaEvent_t ne;
        int rc = check_cuda(cudaEventCreate(&ne));
        if (rc) return rc;
        p->ev_pool.push_back(ne);
    }
    *e = p->ev_pool[p->ev_used++];
    return SFFT4_OK;
}

int prof_begin(sfft4_plan_s* p, cudaStream_t st, cudaEvent_t* a) {
    if (!p->o.profile) return SFFT4_OK;
    int rc = next_event(p, a);
    if (rc) return rc;
    return check_cuda(cudaEventRecord(*a, st));
}

int prof_end(sfft4_plan_s* p, cudaStream_t st, cudaEvent_t a, int kind, int64_t samples, int launches) {
    if (!p->o.profile) return SFFT4_OK;
    cudaEvent_t b;
    int rc = next_event(p, &b);
    if (rc) return rc;
    rc = check_cuda(cudaEventRecord(b, st));
    if (rc) return rc;
    p->prof.push_back({a, b, kind, samples, launches});
    return SFFT4_OK;
}

// Per device, once: the dynamic shared-memory limits of every kernel.  Host threads may make
// their first execute on a device at the same time, so the flag is atomic and the set-up runs
// under a mutex (a failed set-up is retried by the next call).
static std::atomic<bool> g_configured[64];
static std::mutex g_configure_mu;

int configure_kernels() {
    int dev = 0;
    int rc0 = check_cuda(cudaGetDevice(&dev));
    if (rc0) return rc0;
    if (dev < 0 || dev >= 64) return SFFT4_ECUDA;
    if (g_configured[dev].load(std::memory_order_acquire)) return SFFT4_OK;
    std::lock_guard<std::mutex> lk(g_configure_mu);
    if (g_configured[dev].load(std::memory_order_relaxed)) return SFFT4_OK;
    int rc = SFFT4_OK;
    const void* folds[] = {(const void*)k_fold<1>, (const void*)k_fold<2>, (const void*)k_fold<3>,
                           (const void*)k_fold<4>, (const void*)k_fold<5>, (const void*)k_fold<6>,
                           (const void*)k_fold<7>, (const void*)k_fold<8>};
    const void* folds_m[] = {(const void*)k_fold_multi<1>, (const void*)k_fold_multi<2>,
                             (const void*)k_fold_multi<3>, (const void*)k_fold_multi<4>,
                             (const void*)k_fold_multi<5>, (const void*)k_fold_multi<6>,
                             (const void*)k_fold_multi<7>, (const void*)k_fold_multi<8>};
    for (const void* f : folds)
        if (!rc) rc = check_cuda(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kFoldSmemMax));
    for (const void* f : folds_m)
        if (!rc) rc = check_cuda(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kFoldSmemMax));
    const void* folds_s[] = {(const void*)k_fold_sig<1>, (const void*)k_fold_sig<2>,
                             (const void*)k_fold_sig<3>, (const void*)k_fold_sig<4>,
                             (const void*)k_fold_sig<5>, (const void*)k_fold_sig<6>,
                             (const void*)k_fold_sig<7>, (const void*)k_fold_sig<8>};
    for (const void* f : folds_s)
        if (!rc) rc = check_cuda(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kFoldSmemMax));
    const void* decs_m[] = {(const void*)k_decode_multi<8>, (const void*)k_decode_multi<16>,
                            (const void*)k_decode_multi<64>};
    for (const void* f : decs_m)
        if (!rc) rc = check_cuda(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)decode_smem(kBMax)));
    if (!rc) rc = check_cuda(cudaFuncSetAttribute(k_finalize_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  8 * kKMax));
    if (!rc) rc = check_cuda(cudaFuncSetAttribute(k_decode<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)decode_smem(kBMax)));
    if (!rc) rc = check_cuda(cudaFuncSetAttribute(k_decode<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)decode_smem(kBMax)));
    if (!rc) rc = check_cuda(cudaFuncSetAttribute(k_decode<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)decode_smem(kBMax)));
    const void* decs_p[] = {(const void*)k_decode_chain<8>, (const void*)k_decode_chain<16>,
                            (const void*)k_decode_chain<64>, (const void*)k_decode_chain_uniform<8>,
                            (const void*)k_decode_chain_uniform<16>, (const void*)k_decode_chain_uniform<64>};
    for (const void* f : decs_p)
        if (!rc) rc = check_cuda(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)decode_smem(kBMax)));
    const void* decs_c[] = {(const void*)k_decode_cluster<8>, (const void*)k_decode_cluster<16>,
                            (const void*)k_decode_cluster<64>};
    for (const void* f : decs_c) {
        if (!rc) rc = check_cuda(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)decode_smem(kBMax)));
        if (!rc) rc = check_cuda(cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    }
    if (!rc) rc = check_cuda(cudaFuncSetAttribute(k_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  8 * kKMax));
    if (!rc) rc = configure_dft_tc();
    if (!rc) g_configured[dev].store(true, std::memory_order_release);
    return rc;
}

int join_slot0(sfft4_plan_s* p, cudaStream_t st) {
    return (p->async_used & 1) ? check_cuda(cudaStreamWaitEvent(st, p->ev_done[0], 0)) : SFFT4_OK;
}

int mark_sync(sfft4_plan_s* p, cudaStream_t st) {
    if (!p->ev_sync) {
        const int rc = check_cuda(cudaEventCreateWithFlags(&p->ev_sync, cudaEventDisableTiming));
        if (rc) return rc;
    }
    const int rc = check_cuda(cudaEventRecord(p->ev_sync, st));
    if (!rc) p->sync_pending = true;
    return rc;
}

// async_depth workspaces used in turn: this plan's (slot 0) and peer plans of the same
// transform (slots 1..), each on its own stream; slot s's previous execute is ahead on that
// stream, so that many batches can be in flight.
int async_begin(sfft4_plan_s* p, cudaStream_t caller, sfft4_plan_s** w, cudaStream_t* as) {
    int rc = SFFT4_OK;
    // streams and events first (kept if a peer fails, and made again only where missing),
    // then the peers; a peer is stored only once it exists
    for (int s = 0; s < kAsyncDepth && !rc; ++s) {
        if (!p->astream[s]) rc = check_cuda(cudaStreamCreateWithFlags(&p->astream[s], cudaStreamNonBlocking));
        if (!rc && !p->ev_in[s]) rc = check_cuda(cudaEventCreateWithFlags(&p->ev_in[s], cudaEventDisableTiming));
        if (!rc && !p->ev_done[s]) rc = check_cuda(cudaEventCreateWithFlags(&p->ev_done[s], cudaEventDisableTiming));
    }
    if (rc) return rc;
    const int depth = async_depth(p->grp != nullptr);
    for (int i = 0; i < depth - 1; ++i) {
        if (p->peer[i]) continue;
        sfft4_plan_s* peer = nullptr;
        if (p->grp)
            rc = sfft4_plan_batched(&peer, (int32_t)p->bN.size(), p->bN.data(), p->bK.data(),
                                    p->bB1.empty() ? nullptr : p->bB1.data(), p->l, p->bq, p->seed, &p->bopts);
        else
            rc = sfft4_plan(&peer, p->N, p->K, p->l, (double)p->qn / kQDen, p->seed, &p->o);
        if (rc) return rc;
        p->peer[i] = peer;
    }
    const int s = p->async_next;
    *w = s ? p->peer[s - 1] : p;
    *as = p->astream[s];
    rc = check_cuda(cudaEventRecord(p->ev_in[s], caller));
    if (!rc) rc = check_cuda(cudaStreamWaitEvent(*as, p->ev_in[s], 0));
    // slot 0 is the plan's own workspace: also wait for the latest synchronous execute on it,
    // which may have been issued on another stream than `caller`
    if (!rc && s == 0 && p->sync_pending) rc = check_cuda(cudaStreamWaitEvent(*as, p->ev_sync, 0));
    return rc;
}

int async_end(sfft4_plan_s* p, cudaStream_t as) {
    const int s = p->async_next;
    const int rc = check_cuda(cudaEventRecord(p->ev_done[s], as));
    if (rc) return rc;
    p->async_used |= 1 << s;
    p->async_next = (s + 1) % async_depth(p->grp != nullptr);
    return SFFT4_OK;
}

int graph_run(sfft4_plan_s* p, const uint64_t key[8], cudaStream_t st,
              int (*body)(sfft4_plan_s*, const void*, cudaStream_t), const void* ctx) {
    int rc = configure_kernels();
    if (rc) return rc;
    if (!p->o.graph || p->o.profile || p->o.trace) return body(p, ctx, st);
    if (p->gexec && memcmp(key, p->gkey, sizeof(p->gkey)) == 0) return check_cuda(cudaGraphLaunch(p->gexec, st));
    if (p->gexec) {
        rc = check_cuda(cudaGraphExecDestroy(p->gexec));
        p->gexec = nullptr;
        if (rc) return rc;
    }
    if (!p->gstream) {
        rc = check_cuda(cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking));
        if (rc) return rc;
    }
    rc = check_cuda(cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal));
    if (rc) return rc;
    rc = body(p, ctx, p->gstream);
    cudaGraph_t g = nullptr;
    const int rc_end = check_cuda(cudaStreamEndCapture(p->gstream, &g));
    if (!rc) rc = rc_end;
    if (!rc) rc = check_cuda(cudaGraphInstantiate(&p->gexec, g, 0));
    if (g) cudaGraphDestroy(g);
    if (rc) {
        p->gexec = nullptr;
        return rc;
    }
    memcpy(p->gkey, key, sizeof(p->gkey));
    return check_cuda(cudaGraphLaunch(p->gexec, st));
}

}  // namespace sfft4

using namespace sfft4;

namespace {
struct RunArgs {
    int nsig;
    const float2* x;
    int64_t x_stride;
    int64_t* idx;
    sfft4_c128* val;
    int64_t* nfound;
    int8_t* votes;
};

int run_body(sfft4_plan_s* p, const void* ctx, cudaStream_t st) {
    const RunArgs& r = *(const RunArgs*)ctx;
    const int nsig = r.nsig;
    const float2* x = r.x;
    const int64_t x_stride = r.x_stride;
    const size_t ni = p->iters.size();
    // Bucketization of every iteration on the caller's stream; the decode chain on the plan's
    // decode stream, iteration m after its bucket arrays exist (ev[1 + m]) and after decode
    // m - 1 (stream order).  The bucketization never reads the found set.
    cudaStream_t ds = p->dstream;
    int rc = launch_reset(p, nsig, st);
    if (!rc) rc = check_cuda(cudaEventRecord(p->ev[0], st));
    if (!rc) rc = check_cuda(cudaStreamWaitEvent(ds, p->ev[0], 0));
    if (rc) return rc;
    const int64_t rb = (int64_t)p->R_max * p->B_max;
    // signal-major order: one fold launch for every iteration, then the DFTs iteration by
    // iteration (the decode of iteration m starts after its own DFT)
    const bool sig_major = !p->sm_fold.empty();
    // BF16X3 after the signal-major fold: the DFTs of all iterations in grouped launches
    // (the tensor-core DFT holds whole SMs; two launches instead of one or two per iteration)
    const bool all_dft = sig_major && p->uall;
    if (sig_major) {
        rc = launch_fold_signal_major(p, nsig, x, x_stride, st);
        if (rc) return rc;
    }
    if (all_dft) {
        std::vector<DftStrided> sets(ni);
        for (size_t mi = 0; mi < ni; ++mi) {
            const IterHost& ih = p->iters[mi];
            const Window& w = p->wins[ih.win];
            sets[mi] = DftStrided{ih.d.B, ih.d.R, nsig, p->zall + p->yoff[mi], p->ytot, p->uall + p->yoff[mi],
                                  p->ytot, p->y + p->yoff[mi], p->ytot, w.dA1, w.dA2, w.tw4};
        }
        cudaEvent_t ev = nullptr;
        rc = prof_begin(p, st, &ev);
        if (!rc) rc = launch_dft_tc_strided(sets.data(), (int)ni, p->status, p->sm_count, st);
        std::vector<int> Bs(ni);
        for (size_t mi = 0; mi < ni; ++mi) Bs[mi] = (int)p->iters[mi].d.B;
        if (!rc) rc = prof_end(p, st, ev, kProfFft, 0, dft_tc_launches(Bs.data(), (int)ni));
        if (!rc) rc = check_cuda(cudaEventRecord(p->ev[1], st));
        if (!rc) rc = check_cuda(cudaStreamWaitEvent(ds, p->ev[1], 0));
        if (rc) return rc;
    }
    // persistent decode: every iteration's bucket arrays first, then one decode launch
    const bool chain = decode_chain_used(p, nsig);
    for (size_t mi = 0; mi < ni; ++mi) {
        float2* ym = p->y + p->yoff[mi];
        if (!all_dft) {
            rc = sig_major ? launch_iter_dft(p, (int)mi, nsig, p->zall + p->yoff[mi], p->ytot, ym, p->ytot, st)
                           : launch_bucketize(p, (int)mi, nsig, x, x_stride, 0, ym, p->ytot, st);
            if (!rc && !chain) rc = check_cuda(cudaEventRecord(p->ev[1 + mi], st));
            if (!rc && !chain) rc = check_cuda(cudaStreamWaitEvent(ds, p->ev[1 + mi], 0));
            if (rc) return rc;
        }
        if (chain) continue;
        const IterDev& d = p->iters[mi].d;
        const int64_t ts = p->o.trace_signal;  // the traced signal's workspace blocks
        if (p->o.trace) {
            rc = check_cuda(cudaMemcpyAsync(p->trace_y + mi * rb, ym + ts * p->ytot, (size_t)d.R * d.B * sizeof(float2),
                                            cudaMemcpyDeviceToDevice, ds));
            if (rc) return rc;
        }
        rc = launch_decode(p, (int)mi, nsig, ds);
        if (rc) return rc;
        if (p->o.trace) {
            rc = check_cuda(cudaMemcpyAsync(p->trace_F + mi, p->F + ts, sizeof(int32_t), cudaMemcpyDeviceToDevice, ds));
            if (!rc) rc = check_cuda(cudaMemcpyAsync(p->trace_ff + mi * p->Fcap, p->ff + ts * p->Fcap,
                                                     p->Fcap * sizeof(int32_t), cudaMemcpyDeviceToDevice, ds));
            if (!rc) rc = check_cuda(cudaMemcpyAsync(p->trace_fv + mi * p->Fcap, p->fv + ts * p->Fcap,
                                                     p->Fcap * sizeof(double2), cudaMemcpyDeviceToDevice, ds));
            if (!rc) rc = check_cuda(cudaMemcpyAsync(p->trace_votes + mi * p->Fcap, p->fvotes + ts * p->Fcap, p->Fcap,
                                                     cudaMemcpyDeviceToDevice, ds));
            if (rc) return rc;
        }
    }
    if (chain) {
        if (!all_dft) {
            rc = check_cuda(cudaEventRecord(p->ev[1], st));
            if (!rc) rc = check_cuda(cudaStreamWaitEvent(ds, p->ev[1], 0));
        }
        if (!rc) rc = launch_decode_chain_uniform(p, nsig, ds);
        if (rc) return rc;
    }
    rc = launch_finalize(p, nsig, r.idx, r.val, r.nfound, r.votes, ds);
    if (!rc) rc = check_cuda(cudaEventRecord(p->ev[1 + ni], ds));
    if (!rc) rc = check_cuda(cudaStreamWaitEvent(st, p->ev[1 + ni], 0));
    return rc;
}

int run(sfft4_plan_s* p, int nsig, const float2* x, int64_t x_stride, int64_t* idx,
        sfft4_c128* val, int64_t* nfound, int8_t* votes, cudaStream_t st) {
    if (p->grp) return SFFT4_ESTATE;
    if (p->o.trace && p->o.trace_signal >= nsig) return SFFT4_EINVAL;
    const RunArgs r{nsig, x, x_stride, idx, val, nfound, votes};
    const uint64_t key[8] = {p->in_async ? 3u : 1u, (uint64_t)nsig, (uint64_t)(uintptr_t)x, (uint64_t)x_stride,
                             (uint64_t)(uintptr_t)idx, (uint64_t)(uintptr_t)val,
                             (uint64_t)(uintptr_t)nfound, (uint64_t)(uintptr_t)votes};
    int rc = graph_run(p, key, st, run_body, &r);
    if (!rc) {
        p->executed = true;
        ++p->n_executes;
        p->n_transforms += nsig;
        p->last_nsig = nsig;
    }
    return rc;
}
}  // namespace

namespace sfft4 {
int run_execute(sfft4_plan_s* p, int nsig, const float2* x, int64_t x_stride, int64_t* idx,
                sfft4_c128* val, int64_t* nfound, int8_t* votes, cudaStream_t st) {
    return run(p, nsig, x, x_stride, idx, val, nfound, votes, st);
}
}  // namespace sfft4

extern "C" {

int sfft4_execute(sfft4_plan_t p, const void* x_dev, int64_t* idx_dev, sfft4_c128* val_dev,
                  int64_t* nfound_dev, int8_t* votes_dev, void* stream) {
    if (!p || !x_dev || !idx_dev || !val_dev || !nfound_dev) return SFFT4_EINVAL;
    int rc = join_slot0(p, (cudaStream_t)stream);
    if (!rc) rc = run(p, 1, (const float2*)x_dev, p->N, idx_dev, val_dev, nfound_dev, votes_dev,
                      (cudaStream_t)stream);
    if (!rc) rc = mark_sync(p, (cudaStream_t)stream);
    return rc;
}

int sfft4_execute_batched_async(sfft4_plan_t p, int32_t nsig, const void* x_dev, int64_t x_stride,
                                int64_t* idx_dev, sfft4_c128* val_dev, int64_t* nfound_dev,
                                int8_t* votes_dev, void* stream) {
    if (!p || !x_dev || !idx_dev || !val_dev || !nfound_dev) return SFFT4_EINVAL;
    if (p->grp || p->o.trace) return SFFT4_ESTATE;
    if (nsig < 1 || nsig > p->o.max_batch || x_stride < p->N) return SFFT4_EINVAL;
    sfft4_plan_s* w = nullptr;
    cudaStream_t as = nullptr;
    int rc = async_begin(p, (cudaStream_t)stream, &w, &as);
    if (!rc) {
        w->in_async = true;
        rc = run(w, nsig, (const float2*)x_dev, x_stride, idx_dev, val_dev, nfound_dev, votes_dev, as);
        w->in_async = false;
    }
    if (!rc) rc = async_end(p, as);
    return rc;
}

int sfft4_wait(sfft4_plan_t p, void* stream) {
    if (!p) return SFFT4_EINVAL;
    for (int s = 0; s < kAsyncDepth; ++s)
        if ((p->async_used >> s) & 1) {
            const int rc = check_cuda(cudaStreamWaitEvent((cudaStream_t)stream, p->ev_done[s], 0));
            if (rc) return rc;
        }
    return SFFT4_OK;
}

int sfft4_execute_batched(sfft4_plan_t p, int32_t nsig, const void* x_dev, int64_t x_stride,
                          int64_t* idx_dev, sfft4_c128* val_dev, int64_t* nfound_dev,
                          int8_t* votes_dev, void* stream) {
    if (!p || !x_dev || !idx_dev || !val_dev || !nfound_dev) return SFFT4_EINVAL;
    if (p->grp) return SFFT4_ESTATE;
    if (nsig < 1 || nsig > p->o.max_batch || x_stride < p->N) return SFFT4_EINVAL;
    int rc = join_slot0(p, (cudaStream_t)stream);
    if (!rc) rc = run(p, nsig, (const float2*)x_dev, x_stride, idx_dev, val_dev, nfound_dev, votes_dev,
                      (cudaStream_t)stream);
    if (!rc) rc = mark_sync(p, (cudaStream_t)stream);
    return rc;
}

int sfft4_bucketize(sfft4_plan_t p, const void* x_dev, int32_t signal, int32_t m, void* y_dev,
                    void* stream) {
    if (!p || !x_dev || !y_dev || signal < 0 || m < 1 || m > (int32_t)p->iters.size())
        return p && p->grp ? SFFT4_ESTATE : SFFT4_EINVAL;
    const IterDev& d = p->iters[m - 1].d;
    int rc = join_slot0(p, (cudaStream_t)stream);  // the plan's own workspace
    if (!rc) rc = launch_bucketize(p, m - 1, 1, (const float2*)x_dev, p->N, signal, (float2*)y_dev,
                                   (int64_t)d.R * d.B, (cudaStream_t)stream);
    if (!rc) rc = mark_sync(p, (cudaStream_t)stream);
    return rc;
}

int sfft4_stats(sfft4_plan_t p, sfft4_run_stats* out) {
    if (!p || !out) return SFFT4_EINVAL;
    memset(out, 0, sizeof(*out));
    out->executes = p->n_executes;
    out->transforms = p->n_transforms;
    for (const sfft4_plan_s* q : p->peer)
        if (q) {
            out->executes += q->n_executes;
            out->transforms += q->n_transforms;
        }
    out->last_nsig = p->last_nsig;
    std::vector<FinalJob> jobs;
    if (p->grp) {
        int n = 0, kern = 0;
        int64_t samples = 0;
        group_final_jobs(p->grp, &n, &samples, &kern);
        out->samples_per_execute = samples;
        out->iterations = (int32_t)group_levels(p->grp);
        out->kernels_per_execute = kern;
    } else {
        out->samples_per_execute = p->samples * p->last_nsig;
        out->iterations = (int32_t)p->iters.size();
        out->kernels_per_execute = uniform_kernels(p, p->last_nsig > 0 ? p->last_nsig : p->o.max_batch);
        for (int s = 0; s < p->last_nsig; ++s)
            jobs.push_back(FinalJob{p->F + s, p->ff + (int64_t)s * p->Fcap, p->fv + (int64_t)s * p->Fcap,
                                    p->fvotes + (int64_t)s * p->Fcap, p->Fcap, p->K});
    }
    if (!p->executed) return SFFT4_OK;
    int rc = check_cuda(cudaDeviceSynchronize());
    if (rc) return rc;
    const FinalJob* djobs = nullptr;
    FinalJob* tmp = nullptr;
    int nj = 0;
    if (p->grp) {
        int64_t samples;
        int kern;
        djobs = group_final_jobs(p->grp, &nj, &samples, &kern);
    } else {
        nj = (int)jobs.size();
        rc = check_cuda(cudaMalloc(&tmp, jobs.size() * sizeof(FinalJob)));
        if (!rc) rc = check_cuda(cudaMemcpy(tmp, jobs.data(), jobs.size() * sizeof(FinalJob), cudaMemcpyHostToDevice));
        djobs = tmp;
    }
    unsigned long long* dh = nullptr;
    if (!rc) rc = check_cuda(cudaMalloc(&dh, (SFFT4_MAX_VOTES + 1) * sizeof(unsigned long long)));
    if (!rc) rc = check_cuda(cudaMemset(dh, 0, (SFFT4_MAX_VOTES + 1) * sizeof(unsigned long long)));
    if (!rc) rc = launch_votes_hist(djobs, nj, dh, 0);
    unsigned long long hh[SFFT4_MAX_VOTES + 1] = {0};
    if (!rc) rc = check_cuda(cudaMemcpy(hh, dh, sizeof(hh), cudaMemcpyDeviceToHost));
    cudaFree(dh);
    cudaFree(tmp);
    if (rc) return rc;
    for (int v = 0; v <= SFFT4_MAX_VOTES; ++v) {
        out->votes_hist[v] = (int64_t)hh[v];
        out->last_found += (int64_t)hh[v];
    }
    return SFFT4_OK;
}

int sfft4_sync_status(sfft4_plan_t p) {
    if (!p) return SFFT4_EINVAL;
    int rc = check_cuda(cudaDeviceSynchronize());
    if (rc) return rc;
    int32_t st = 0;
    rc = check_cuda(cudaMemcpy(&st, p->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (rc) return rc;
    if (st) {
        rc = check_cuda(cudaMemset(p->status, 0, sizeof(int32_t)));
        if (rc) return rc;
        return SFFT4_ETIMEOUT;
    }
    return SFFT4_OK;
}

int sfft4_inject_status(sfft4_plan_t p, int32_t value) {
    if (!p || !p->status) return SFFT4_EINVAL;
    return check_cuda(cudaMemcpy(p->status, &value, sizeof(int32_t), cudaMemcpyHostToDevice));
}

int sfft4_profile_get(sfft4_plan_t p, sfft4_profile* out, int32_t reset) {
    if (!p || !out) return SFFT4_EINVAL;
    if (!p->o.profile) return SFFT4_ESTATE;
    for (sfft4_plan_s* pp : p->peer) {
        if (!pp) continue;
        // the other workspaces' launches (asynchronous executes) count with this plan's
        sfft4_profile q;
        int rc = sfft4_profile_get(pp, &q, 1);
        if (rc) return rc;
        p->prof_tot.fold_launches += q.fold_launches;
        p->prof_tot.fold_ms += q.fold_ms;
        p->prof_tot.fold_samples += q.fold_samples;
        p->prof_tot.fft_launches += q.fft_launches;
        p->prof_tot.fft_ms += q.fft_ms;
        p->prof_tot.decode_launches += q.decode_launches;
        p->prof_tot.decode_ms += q.decode_ms;
        p->prof_tot.finalize_launches += q.finalize_launches;
        p->prof_tot.finalize_ms += q.finalize_ms;
    }
    for (auto& r : p->prof) {
        int rc = check_cuda(cudaEventSynchronize(r.b));
        if (rc) return rc;
        float ms = 0.f;
        rc = check_cuda(cudaEventElapsedTime(&ms, r.a, r.b));
        if (rc) return rc;
        switch (r.kind) {
            case kProfFold: p->prof_tot.fold_launches++; p->prof_tot.fold_ms += ms;
                            p->prof_tot.fold_samples += r.samples; break;
            case kProfFft: p->prof_tot.fft_launches += r.launches; p->prof_tot.fft_ms += ms; break;
            case kProfDecode: p->prof_tot.decode_launches++; p->prof_tot.decode_ms += ms; break;
            default: p->prof_tot.finalize_launches++; p->prof_tot.finalize_ms += ms; break;
        }
    }
    p->prof.clear();
    p->ev_used = 0;
    *out = p->prof_tot;
    if (reset) p->prof_tot = sfft4_profile{};
    return SFFT4_OK;
}

int sfft4_trace_get(sfft4_plan_t p, int32_t m, void* y_host, int64_t cap, int64_t* f_host,
                    sfft4_c128* v_host, int8_t* votes_host, int64_t* nfound) {
    if (!p || m < 1 || m > (int32_t)p->iters.size()) return SFFT4_EINVAL;
    if (!p->o.trace || !p->executed) return SFFT4_ESTATE;
    int rc = check_cuda(cudaDeviceSynchronize());
    if (rc) return rc;
    const IterDev& d = p->iters[m - 1].d;
    const int64_t rb = (int64_t)p->R_max * p->B_max;
    if (y_host) {
        rc = check_cuda(cudaMemcpy(y_host, p->trace_y + (m - 1) * rb, (size_t)d.R * d.B * sizeof(float2),
                                   cudaMemcpyDeviceToHost));
        if (rc) return rc;
    }
    int32_t F = 0;
    rc = check_cuda(cudaMemcpy(&F, p->trace_F + (m - 1), sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (rc) return rc;
    if (nfound) *nfound = F;
    int64_t nc = std::min<int64_t>(F, cap);
    if (nc > 0) {
        std::vector<int32_t> f32(nc);
        std::vector<double2> v(nc);
        std::vector<int8_t> vt(nc);
        rc = check_cuda(cudaMemcpy(f32.data(), p->trace_ff + (m - 1) * p->Fcap, nc * sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (!rc) rc = check_cuda(cudaMemcpy(v.data(), p->trace_fv + (m - 1) * p->Fcap, nc * sizeof(double2), cudaMemcpyDeviceToHost));
        if (!rc) rc = check_cuda(cudaMemcpy(vt.data(), p->trace_votes + (m - 1) * p->Fcap, nc, cudaMemcpyDeviceToHost));
        if (rc) return rc;
        for (int64_t i = 0; i < nc; ++i) {
            if (f_host) f_host[i] = f32[i];
            if (v_host) { v_host[i].re = v[i].x; v_host[i].im = v[i].y; }
            if (votes_host) votes_host[i] = vt[i];
        }
    }
    return SFFT4_OK;
}

}  // extern "C"
