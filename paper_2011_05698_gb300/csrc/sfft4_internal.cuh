// Internal definitions of the sFFT4.0 GB300 library: plan structures shared by the host
// planner and the kernels, and small device helpers (Philox, modular inverse, fixed-point
// phases).  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "sfft4.h"

namespace sfft4 {

constexpr int kMaxRounds = SFFT4_MAX_ROUNDS;  // R = S + 1 <= 64 rounds per iteration
constexpr int kFoldRG = 8;                    // rounds accumulated per fold launch group
constexpr int kFoldGroupMax = 3;              // rounds per fold group the planner forms (measured
                                              // against 2, 4, 5, 6 and 7 on N = 2^22, K = 1000)
constexpr int kFoldGroupMaxBatched = 6;       // the same for sfft4_plan_batched (a 512-signal batch
                                              // of N = 2^16..2^22: 189-194 K transforms/s
                                              // pipelined with 6, 178 K with 4, 163-167 K with 3)
constexpr int kMaxSeg = 2 * kFoldRG + 2;      // t-segments of one fold group
constexpr int kQDen = 256;                    // q = q_n / 256
constexpr int kBMin = 16;
constexpr int kBMax = 4096;
constexpr int kKMax = 4096;
constexpr int kDecodeThreads = 512;     // two decode CTAs per SM
constexpr int kAsyncDepth = 3;          // most workspaces of the asynchronous executes
// Batches in flight: two for a uniform batch (a third would run two signal-major folds at
// once and spoil their L2 reuse: 54 K against 79 K transforms/s at N = 2^22, K = 1000), three
// for a batch of uneven signals (folded level by level; its step is its decode chain, and
// two chains overlap: 78 K against 66 K transforms/s on the 512-signal workload).
inline int async_depth(bool uneven) { return uneven ? 3 : 2; }
constexpr int kFoldSmemMax = 32 * 1024;      // per-copy sums of one fold CTA (8 rounds x 512 threads)

// Rounds [r0, r0 + nr) of one iteration that one fold launch accumulates, and the
// t-segments covering the union of their windows [tau_s - h, tau_s + h]; within a segment
// the set of covering rounds (mask, bit s - r0) is constant.
struct FoldGroup {
    int32_t r0, nr, nseg;
    int32_t P;                 // copies per residue (threads per slot)
    int64_t t0[kMaxSeg], t1[kMaxSeg];  // half-open [t0, t1)
    uint32_t mask[kMaxSeg];
    int64_t unique;            // samples this group reads
};

// Device-resident parameters of one iteration (read by the fold, FFT and decode kernels).
struct IterDev {
    int32_t m, B, logB, S, R, n_c, h, logL;
    int64_t L;
    int64_t Lbar[kMaxRounds];          // levels 1..S at index 0..S-1
    int64_t tau[kMaxRounds + 1];       // tau_0 = 0 .. tau_S
    uint32_t H[kMaxRounds];            // vote thresholds, levels 1..S at index 0..S-1
    uint64_t W[kMaxRounds];            // phase span (Lbar_s tau_s) << (32 - n) of level s
    float jscale[kMaxRounds];          // l / W (block levels), 1 / W (final level)
    uint32_t Cj[kMaxRounds][32];       // block centre offsets ((2j+1) W + l) / (2l)
    int32_t Dj[kMaxRounds][32];        // region shifts floor((2jQ - q_n) Lbar_s / (2lQ))
    const float* G;                    // w = 2h + 1 window coefficients G_{-h..h}
    const float* Ghat;                 // G'^_k for k = 0..3L/2
    const float2* tw;                  // e^{-2 pi i k / B}, k < B/2
};

struct Window {
    int64_t N = 0;
    int32_t B, h;
    int64_t L;
    float* G = nullptr;        // device, 2h + 1
    float* Ghat = nullptr;     // device, 3L/2 + 1
    float2* tw = nullptr;      // device, B/2
    // tensor-core DFT (precision SFFT4_BF16X3): split DFT matrices of both stages, twiddles
    unsigned char* dA1 = nullptr;
    unsigned char* dA2 = nullptr;
    float2* tw4 = nullptr;     // device, B
};

struct IterHost {
    IterDev d;
    std::vector<FoldGroup> groups;
    int64_t unique;            // |union_s [tau_s - h, tau_s + h]|
    int32_t win;               // index into plan windows
    int32_t Wj;                // residues per fold CTA
};

// Arguments of one fold launch (uniform batch) or one fold job (batch of different sizes).
struct FoldArgs {
    const float2* x;
    int64_t x_stride;
    float2* z;
    int64_t z_stride;
    uint64_t N, seed;
    int32_t m, signal0, B, logB, Wj, h, w;
    const float* G;
    FoldGroup g;
    int32_t tau[kFoldRG];
};

// Dynamic shared memory of a fold launch of `threads` threads whose jobs have at most rg
// rounds: the per-copy sums of every round (rg x threads float2).
inline size_t fold_smem(int rg, int threads) { return (size_t)rg * threads * 8; }

struct FoldTile {
    int32_t job, slice;
};

// One signal-major fold launch: the (iteration, fold group) jobs it covers, passed in the
// kernel's parameter space (warp-uniform constant loads, no per-CTA copy), job j owning the
// residue slices start[j] .. start[j + 1] - 1 of each signal's tile range.
constexpr int kSigJobs = 48;
struct SigFoldLaunch {
    const float2* x;
    int64_t x_stride;
    int32_t ntiles, njobs;
    int32_t start[kSigJobs + 1];
    FoldArgs jobs[kSigJobs];
};
struct SigFoldHost {
    SigFoldLaunch L;
    int32_t RG, threads;
    size_t smem;
    int64_t samples;  // per signal
};

// Arguments of one decode launch (uniform batch) or one signal's decode (batch of sizes).
struct DecodeArgs {
    uint64_t N, seed;
    int32_t n, signal0, first, l, qn, min_votes;
    int32_t fine_phase;   // final level's phase in FP64 (two-round location: step 1/N)
    float mag_tol, sig_floor;
    const IterDev* it;
    float2* y;
    int64_t y_stride;
    int32_t* F;
    int32_t* ff;
    double2* fv;
    int8_t* fvotes;
    int64_t Fcap;
    int32_t* hkeys;
    int32_t* hvals;
    int32_t Hlog;
    float* theta;
    int32_t* fxexp;
};

struct FinalJob {
    const int32_t* F;
    const int32_t* ff;
    const double2* fv;
    const int8_t* fvt;
    int64_t Fcap, K;
};

// ------------------------------------------------------------------ device helpers ---
#define SFFT4_HD __host__ __device__ __forceinline__

SFFT4_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Philox4x64-10 (Salmon et al., SC'11): one 4 x 64-bit block for a counter and key.
SFFT4_HD void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    for (int r = 0; r < 10; ++r) {
        uint64_t lo0 = M0 * c[0], hi0 = mulhi64(M0, c[0]);
        uint64_t lo1 = M1 * c[2], hi1 = mulhi64(M1, c[2]);
        uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += W0; k1 += W1;
    }
}

// (sigma, a) of iteration m of signal `signal`: counter (signal, m, 0, 0), key (seed, 0);
// sigma = 2 (r0 mod N/2) + 1 is odd (invertible mod N = 2^n), a = r1 mod N (Section 2.2).
SFFT4_HD void permutation_draw(uint64_t seed, uint64_t signal, uint64_t m, uint64_t N,
                               uint64_t* sigma, uint64_t* a) {
    uint64_t c[4] = {signal, m, 0, 0};
    philox4x64_10(c, seed, 0);
    *sigma = 2 * (c[0] & (N / 2 - 1)) + 1;
    *a = c[1] & (N - 1);
}

// Inverse of an odd sigma modulo 2^64 by Newton's iteration x <- x (2 - sigma x).
SFFT4_HD uint64_t inv_odd64(uint64_t s) {
    uint64_t x = s;  // correct to 3 bits for odd s
    for (int i = 0; i < 5; ++i) x *= 2 - s * x;
    return x;
}

// Distance of two phases held as 2^-32 turns, on the circle.
SFFT4_HD uint32_t circ_dist(uint32_t a, uint32_t b) {
    uint32_t d = a - b;
    uint32_t e = b - a;
    return d < e ? d : e;
}

// floor(a / b) for b > 0 and any sign of a.
SFFT4_HD int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) --q;
    return q;
}

struct Group;  // batch of signals of different sizes (group.cu)

}  // namespace sfft4

// The opaque plan.
struct sfft4_plan_s {
    int64_t N;
    int n;
    int64_t K;
    int32_t l, qn;
    uint64_t seed;
    sfft4_opts o;
    int device;
    std::vector<sfft4::IterHost> iters;
    std::vector<sfft4::Window> wins;
    sfft4::IterDev* iters_dev = nullptr;
    int32_t B_max = 0, R_max = 0;
    int64_t Fcap = 0;           // found entries per signal
    int32_t Hlog = 0;           // log2 of hash slots per signal
    int64_t samples = 0;        // distinct samples per transform
    // workspace for o.max_batch signals
    float2* z = nullptr;        // [sig][R_max][B_max] folded, before the DFT
    float2* y = nullptr;        // [sig][ytot] bucket arrays of every iteration (iteration m at yoff[m])
    std::vector<int64_t> yoff;  // offset of iteration m's R_m x B_m arrays within a signal's block
    int64_t ytot = 0;           // sum over iterations of R_m B_m
    int32_t* F = nullptr;       // [sig] found count
    int32_t* ff = nullptr;      // [sig][Fcap] frequency
    double2* fv = nullptr;      // [sig][Fcap] value
    int8_t* fvotes = nullptr;   // [sig][Fcap]
    int32_t* hkeys = nullptr;   // [sig][2^Hlog] hash keys (frequency or -1)
    int32_t* hvals = nullptr;   // [sig][2^Hlog] entry index
    float2* u = nullptr;        // [sig][R_max][B_max] four-step scratch (BF16X3 DFT)
    // signal-major fold (fold_order SFFT4_FOLD_SIGNAL_MAJOR): one job per (iteration, fold
    // group) with z of iteration m at zall + yoff[m] (per-signal stride ytot); a launch's grid
    // is nsig x ntiles CTAs, the ntiles (job, residue slice) tiles of a signal adjacent
    float2* zall = nullptr;     // [sig][ytot] folded arrays of every iteration
    float2* uall = nullptr;     // [sig][ytot] four-step scratch of every iteration (BF16X3)
    std::vector<sfft4::SigFoldHost> sm_fold;  // launches (more than one past kSigJobs jobs)
    // asynchronous executes (sfft4_execute_batched_async): kAsyncDepth workspaces, this
    // plan's (slot 0) and peer plans' (slots 1..), used in turn on their own streams;
    // ev_done[s] marks slot s's latest execute
    sfft4_plan_s* peer[sfft4::kAsyncDepth - 1] = {};
    std::vector<int64_t> bN, bK;        // sfft4_plan_batched's arguments (to make the peer)
    std::vector<int32_t> bB1;
    double bq = 0;
    sfft4_opts bopts;
    cudaStream_t astream[sfft4::kAsyncDepth] = {};
    cudaEvent_t ev_in[sfft4::kAsyncDepth] = {};
    cudaEvent_t ev_done[sfft4::kAsyncDepth] = {};
    int async_next = 0, async_used = 0;
    // end of the latest synchronous execute (or bucketization) on the plan's own workspace, on
    // the caller's stream; an asynchronous execute that takes slot 0 waits for it
    cudaEvent_t ev_sync = nullptr;
    bool sync_pending = false;
    // host-buffer executes (sfft4_execute_batched_host): device copies of max_batch inputs
    // (dense rows of N) and outputs, allocated by the first such execute on this workspace
    float2* hx = nullptr;
    int64_t* hidx = nullptr;
    sfft4_c128* hval = nullptr;
    int64_t* hnf = nullptr;
    int8_t* hvotes = nullptr;
    // the stagings of consecutive host-buffer executes, one after another on their own stream
    // (the host link stays busy); ev_staged[s] marks slot s's latest staging
    cudaStream_t hstream = nullptr;
    cudaEvent_t ev_staged[sfft4::kAsyncDepth] = {};
    int32_t* status = nullptr;  // 1 when a bounded device wait gave up
    int sm_count = 0;
    // persistent decode of a signal-major batch (opts.batch_exec): every iteration's decode
    // arguments, the queue counter of the launch, its round class and shared memory
    sfft4::DecodeArgs* dec_iters = nullptr;
    bool in_async = false;      // set while an asynchronous execute runs on this workspace
    int32_t* queue = nullptr;
    int32_t dec_rclass = 0;
    size_t dec_smem = 0;
    float* theta = nullptr;     // [sig] candidate floor
    int32_t* fxexp = nullptr;   // [sig] fixed-point exponent of the bucket update
    // trace of signal 0 (opts.trace)
    float2* trace_y = nullptr;      // [iter][R_max][B_max]
    int32_t* trace_F = nullptr;     // [iter]
    int32_t* trace_ff = nullptr;    // [iter][Fcap]
    double2* trace_fv = nullptr;    // [iter][Fcap]
    int8_t* trace_votes = nullptr;  // [iter][Fcap]
    bool executed = false;
    int64_t n_executes = 0, n_transforms = 0;  // counters (sfft4_stats)
    int32_t last_nsig = 0;
    bool owns_tables = true;    // false when the window tables belong to a batch's cache
    sfft4::Group* grp = nullptr;  // set for plans from sfft4_plan_batched
    // CUDA graph of the last captured execute (opts.graph), keyed on its buffers
    cudaStream_t gstream = nullptr;
    // the decode chain runs on its own stream, overlapping the bucketization of later
    // iterations (which does not depend on it); ev[0] forks, ev[1 + m] marks iteration m's
    // bucket arrays, ev.back() joins
    cudaStream_t dstream = nullptr;
    std::vector<cudaEvent_t> ev;
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey[8] = {};
    // profiling (opts.profile): event pairs recorded around launches, by kind
    struct Prof {
        cudaEvent_t a, b;
        int kind;
        int64_t samples;
        int launches;  // kernels launched between a and b
    };
    std::vector<cudaEvent_t> ev_pool;
    std::vector<Prof> prof;
    size_t ev_used = 0;
    sfft4_profile prof_tot{};
};

namespace sfft4 {
// Implemented in kernels.cu.
int build_window_tables(sfft4_plan_s* p, Window* w, double delta);
int launch_bucketize(sfft4_plan_s* p, int m_index, int nsig, const float2* x, int64_t x_stride,
                     int32_t signal0, float2* y_out, int64_t y_sig_stride, cudaStream_t st);
int launch_decode(sfft4_plan_s* p, int m_index, int nsig, cudaStream_t st);
// Whether an execute of nsig signals decodes in one persistent launch (opts.batch_exec
// persistent, signal-major fold, one CTA per signal, no trace), and that launch.
bool decode_chain_used(const sfft4_plan_s* p, int nsig);
int launch_decode_chain_uniform(sfft4_plan_s* p, int nsig, cudaStream_t st);
int build_decode_chain(sfft4_plan_s* p);
int launch_finalize(sfft4_plan_s* p, int nsig, int64_t* idx, sfft4_c128* val, int64_t* nfound,
                    int8_t* votes, cudaStream_t st);
int launch_reset(sfft4_plan_s* p, int nsig, cudaStream_t st);
FoldArgs make_fold_args(const sfft4_plan_s* p, int mi, const FoldGroup& g, size_t* smem_out);
DecodeArgs make_decode_args(const sfft4_plan_s* p, int mi);
size_t decode_smem_bytes(int B);
int configure_kernels();
int build_signal_major_fold(sfft4_plan_s* p);
// Workspace and stream of the next asynchronous execute (makes the peer plan on first use),
// after the execute reads its inputs behind the work queued on `caller`; async_end marks it.
int async_begin(sfft4_plan_s* p, cudaStream_t caller, sfft4_plan_s** w, cudaStream_t* as);
int async_end(sfft4_plan_s* p, cudaStream_t as);
// One execute of nsig signals on workspace p (stream st): the body of every execute entry.
int run_execute(sfft4_plan_s* p, int nsig, const float2* x, int64_t x_stride, int64_t* idx,
                sfft4_c128* val, int64_t* nfound, int8_t* votes, cudaStream_t st);
// A synchronous execute waits for the asynchronous one that used the plan's own workspace;
// mark_sync records its end, which the next asynchronous execute in slot 0 waits for.
int join_slot0(sfft4_plan_s* p, cudaStream_t st);
int mark_sync(sfft4_plan_s* p, cudaStream_t st);
int launch_fold_signal_major(sfft4_plan_s* p, int nsig, const float2* x, int64_t x_stride, cudaStream_t st);
int launch_fold_multi(int RG, const FoldArgs* jobs, const FoldTile* tiles, int ntiles,
                      const float2* const* xptrs, int threads, size_t smem, cudaStream_t st);
int launch_fft_multi(const float2* const* zcols, float2* const* ycols, int ncols, int B,
                     const float2* tw, cudaStream_t st);
int launch_decode_multi(int rclass, const DecodeArgs* jobs, const int32_t* list, int n, size_t smem,
                        cudaStream_t st);
int launch_decode_chain(int rclass, const DecodeArgs* jobs, const int32_t* off, const int32_t* len,
                        const int32_t* order, int nsig, int32_t* queue, int grid, size_t smem, cudaStream_t st);
int launch_finalize_multi(const FinalJob* jobs, int nsig, int64_t Kout, int64_t* idx, sfft4_c128* val,
                          int64_t* nfound, int8_t* votes, cudaStream_t st);
int launch_votes_hist(const FinalJob* jobs, int nsig, unsigned long long* hist, cudaStream_t st);
int prof_begin(sfft4_plan_s* p, cudaStream_t st, cudaEvent_t* a);
int prof_end(sfft4_plan_s* p, cudaStream_t st, cudaEvent_t a, int kind, int64_t samples, int launches = 1);
enum { kProfFold = 0, kProfFft = 1, kProfDecode = 2, kProfFinalize = 3 };
int check_cuda(cudaError_t e);
// Runs body(stream) directly, or (opts.graph) replays the graph captured from it for the
// same key, capturing it first on the plan's private stream.
int graph_run(sfft4_plan_s* p, const uint64_t key[8], cudaStream_t st, int (*body)(sfft4_plan_s*, const void*, cudaStream_t),
              const void* ctx);
// Implemented in group.cu.
int build_group_plan(sfft4_plan_s* p, int nsig, const int64_t* N, const int64_t* K, const int32_t* B1, int32_t l,
                     double q, uint64_t seed, const sfft4_opts* opts);
void destroy_group(Group* g);
size_t group_levels(const Group* g);
const FinalJob* group_final_jobs(const Group* g, int* nsig, int64_t* samples, int* kernels);
// Implemented in plan.cu.
// Half-width h of the flat window of B buckets at leakage delta (Eq. 9, the window design of
// a Gaussian of time-domain std s_t = B 4 sqrt2 erfcinv(delta) / (2 pi) truncated at delta):
// h = ceil(s_t sqrt(2 ln(1/delta))); *s_t_out (if not NULL) receives s_t.  The one definition
// every table builder uses.
int64_t window_halfwidth(int64_t B, double delta, double* s_t_out);
int plan_options(int64_t N, int64_t K, int32_t l, double q, const sfft4_opts* opts, sfft4_opts* out,
                 int* qn_out);
int plan_schedule(sfft4_plan_s* p);
int32_t uniform_kernels(const sfft4_plan_s* p, int nsig);
int plan_tables(sfft4_plan_s* p, std::vector<Window>* cache);
// Implemented in dft_tc.cu.
size_t dft_tc_matrix_bytes();
int build_dft_tc_tables(int B, unsigned char* A1, unsigned char* A2, float2* tw4);
int configure_dft_tc();
// One iteration's DFT columns for launch_dft_tc_strided: signal s's R x B arrays at
// z + s z_stride (input), u + s u_stride (four-step scratch), y + s y_stride (output).
struct DftStrided {
    int32_t B, R, nsig;
    const float2* z;
    int64_t z_stride;
    float2* u;
    int64_t u_stride;
    float2* y;
    int64_t y_stride;
    const unsigned char* A1;
    const unsigned char* A2;
    const float2* tw4;
};
int launch_dft_tc_strided(const DftStrided* sets, int nsets, int32_t* status, int sm_count, cudaStream_t st);
int launch_dft_tc(const float2* z, int64_t z_stride, float2* u, int64_t u_stride, float2* y, int64_t y_stride, int nsig,
                  int R, int B, const unsigned char* A1, const unsigned char* A2, const float2* tw4,
                  int32_t* status, int sm_count, cudaStream_t st);
// Columns of one bucket count within a level of a batch of uneven signals (device tables of
// per-column z, u and y base pointers).
struct DftColSet {
    int B;
    const unsigned char* A1;
    const unsigned char* A2;
    const float2* tw4;
    const float2* const* zcols;
    float2* const* ucols;
    float2* const* ycols;
    int64_t ncols;
};
int launch_dft_tc_sets(const DftColSet* sets, int nsets, int32_t* status, int sm_count, cudaStream_t st);
int dft_tc_launches(const int* Bs, int nsets);  // launches launch_dft_tc_sets makes
}  // namespace sfft4
