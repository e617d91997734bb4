/*
 * sfft4.h -- C ABI of the GB300 (sm_103a) sFFT4.0 library.
 *
 * sFFT4.0 is the multiscale flat-window sparse FFT of Li, Jiang and Chen, "On Performance
 * of Multiscale Sparse Fast Fourier Transform Algorithm" (arXiv 2011.05698).  Given a
 * length-N signal whose spectrum is (approximately) K-sparse, it returns K (frequency,
 * value) pairs while reading only a small fraction of the samples.
 *
 * Conventions (Section 2.1, Eq. 1-2): X_f = (1/N) sum_n x_n exp(-2 pi i f n / N); the
 * values returned are these X_f (a unit-magnitude tone x_n = exp(2 pi i f n / N) returns
 * X_f = 1).
 *
 * All entry points return 0 (SFFT4_OK) or a negative SFFT4_E* code; no exception or
 * longjmp crosses the ABI.  Device pointers are caller-owned and must stay valid until the
 * work queued on the given stream has completed.  Execution is asynchronous on the
 * caller's stream (a cudaStream_t passed as void*; NULL = the legacy default stream).
 * A plan is not thread-safe: do not execute one plan concurrently from two host threads
 * or on two streams at once (its workspace is shared by all its executions).  The
 * asynchronous executes (sfft4_execute_batched_async, sfft4_execute_batched_v_async) are the
 * exception: they alternate two (uniform batches) or three (batches of uneven signals)
 * workspaces on the plan's own streams by themselves.
 */
#ifndef SFFT4_H
#define SFFT4_H

#include <stdint.h>

#if defined(__GNUC__)
#define SFFT4_API __attribute__((visibility("default")))
#else
#define SFFT4_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- error codes ---- */
#define SFFT4_OK 0
#define SFFT4_EINVAL (-1)   /* invalid argument (sizes, parameters, null pointers)      */
#define SFFT4_ENOMEM (-2)   /* device or host allocation failed                        */
#define SFFT4_ECUDA (-3)    /* a CUDA runtime call failed (details: sfft4_last_cuda_error) */
#define SFFT4_ESTATE (-4)   /* call not valid in the plan's current state               */
#define SFFT4_ETIMEOUT (-5) /* a bounded device-side wait gave up (see sfft4_sync_status) */

/* ----------------------------------------------------------------- precision ------ */
#define SFFT4_FP32 0        /* window, fold and B-point DFT in FP32 (CUDA cores)         */
#define SFFT4_BF16X3 1      /* B-point DFT as a BF16x3 split-precision complex GEMM on   */
                            /* the tensor cores (tcgen05), FP32 accumulation             */

/* ----------------------------------------------------------------- options -------- */
#define SFFT4_LOC_MULTISCALE 0        /* sfft4_opts.location */
#define SFFT4_LOC_TWO_ROUND 1
#define SFFT4_FOLD_SIGNAL_MAJOR 0     /* sfft4_opts.fold_order */
#define SFFT4_FOLD_ITERATION_MAJOR 1
#define SFFT4_BATCH_PERSISTENT 0      /* sfft4_opts.batch_exec */
#define SFFT4_BATCH_LEVELS 1

typedef struct sfft4_plan_s* sfft4_plan_t;   /* opaque, library-owned */

typedef struct {
    double re, im;
} sfft4_c128;

/* Plan options; a zero field means "default".  Fill with sfft4_opts_default(). */
typedef struct {
    int32_t B1;              /* buckets of iteration 1 (power of two, 16..4096, <= N/64);
                                default pow2ceil(2K) capped at min(4096, N/64), then halved
                                while the window (about 44 B1 samples at delta 1e-8) is wider
                                than N/2                                                   */
    double delta;            /* flat-window leakage delta of Eq. 9; default 1e-8          */
    int32_t precision;       /* SFFT4_FP32 (default) or SFFT4_BF16X3                      */
    int32_t min_votes;       /* levels that must vote to accept; default = all levels     */
    double select_factor;    /* c in n_c = min(B_m, ceil(c max(K_m, 1))); default 2       */
    double sig_floor;        /* candidate floor relative to max |yhat_0|^2 of iteration 1;
                                default 1e-10; negative disables the floor                 */
    double mag_tol;          /* magnitude consistency of a vote; default 0.5              */
    int32_t max_iters;       /* cap on the static schedule length; default 64             */
    int32_t max_batch;       /* most signals one sfft4_execute_batched call may pass;
                                sizes the workspace; with the signal-major fold, max_batch
                                x the fold tiles of one signal must stay below 2^31 (one
                                launch grid), with the iteration-major fold max_batch <= 65535
                                (signals in grid.y), else SFFT4_EINVAL; default 1           */
    int32_t trace;           /* nonzero: keep per-iteration bucket arrays and found sets
                                of signal 0 for sfft4_trace_get (tests); default 0         */
    int32_t profile;         /* nonzero: bracket each kernel launch of an execute with CUDA
                                events on the execution stream (sfft4_profile_get)        */
    int32_t l2_fetch_bytes;  /* L2 fetch granularity hint the plan sets on the calling
                                process's CUDA context (cudaLimitMaxL2FetchGranularity):
                                0 = 64 bytes (measured best for the signal-major fold),
                                32 or 128 = that many bytes, negative = leave the context's
                                limit unchanged                                            */
    int32_t graph;           /* nonzero: the first execute with a given set of buffers and
                                batch size captures its launch sequence as a CUDA graph;
                                later executes with the same buffers replay it (one graph
                                launch).  Ignored when profile or trace is set.  The graph
                                holds the buffer addresses: the caller keeps them valid
                                while the plan may replay it                              */
    int32_t location;        /* SFFT4_LOC_MULTISCALE (default; Section 3.2) or
                                SFFT4_LOC_TWO_ROUND (sFFT3.0-style: rounds tau = 0 and 1, the
                                phase of yhat_1 / yhat_0 is u / N; exactly sparse signals with
                                few collisions; default B1 pow2ceil(8K); N <= 2^20, where FP32
                                bucket arrays resolve its 1/(8N)-turn vote window)          */
    int32_t fold_order;      /* order of the fold work of a batched execute:
                                SFFT4_FOLD_SIGNAL_MAJOR (default): one launch folds every
                                iteration of the batch, the CTAs of one signal's iterations
                                adjacent, so that the random samples the iterations share are
                                read from DRAM once and re-read from L2;
                                SFFT4_FOLD_ITERATION_MAJOR: one launch per iteration group over
                                the whole batch (each signal's samples read once per iteration) */
    int32_t trace_signal;    /* with trace: the batch index of the signal whose per-iteration
                                bucket arrays and found sets sfft4_trace_get returns (0 <=
                                trace_signal < max_batch; an execute of fewer signals than
                                trace_signal + 1 returns SFFT4_EINVAL); default 0           */
    int32_t batch_exec;      /* how an execute of sfft4_plan_batched runs its signals:
                                SFFT4_BATCH_PERSISTENT (default): every (signal, iteration,
                                residue slice) fold tile in one launch, the DFT columns of every
                                iteration grouped by bucket count, and one decode launch of
                                persistent CTAs that take whole signals from a device queue
                                (longest decode chains first) and run their iterations in
                                order; SFFT4_BATCH_LEVELS: level by level (level m = iteration
                                m of every signal that has one), the decode chain on a second
                                stream.  The results are identical                          */
    int32_t fold_residues;   /* fold tile shape: residues mod B per fold CTA (16, 32 or 64,
                                at most B); default 64.  It sets the copies per residue and
                                so the order of the fold's copy sums (results agree to FP32
                                rounding, not bit for bit)                                  */
    int32_t fold_rounds;     /* fold tile shape: most rounds one fold CTA accumulates (1..8;
                                an iteration's rounds are split into balanced groups of at
                                most this many); default 3, 6 for sfft4_plan_batched.  It
                                regroups the tiles only: every round's samples are still
                                added in the same order.  An autotuner may pick both per
                                (N, K)                                                      */
    int32_t decode_cluster;  /* CTAs that decode one signal (a thread-block cluster of 1, 2,
                                4, 8 or 16 CTAs sharing the update's buckets and the
                                candidates); 0 (default) = the largest power of two up to 4
                                with which the execute's decode CTAs fit on the SMs (up to
                                38 signals: 4; up to 76: 2; more: 1).  The results do not
                                depend on it                                         */
} sfft4_opts;

/* Fills *opts with the defaults above.  Returns SFFT4_EINVAL if opts is NULL. */
SFFT4_API int sfft4_opts_default(sfft4_opts* opts);

/*
 * sfft4_plan -- build the static plan of one transform size (Section 3.1, Lemma 2).
 *   N     transform length, a power of two in [2^8, 2^30]
 *   K     sparsity, 1 <= K <= min(4096, N/64)
 *   l     multiscale parameter (blocks per level, Section 3.2), 2 <= l <= 32
 *   q     extension parameter (Section 3.2), 0 <= q, l > q + 1; quantised to q_n/256
 *   seed  key of the Philox4x64-10 draws of sigma and the per-iteration offset: signal i of a
 *         batch, iteration m uses counter (i, m, 0, 0) and key (seed, 0)
 *   opts  may be NULL (all defaults)
 * On success *out owns device tables (window G and its spectrum for every bucket count of
 * the schedule, FFT twiddles) and workspace for opts->max_batch signals.  The window tables
 * are generated by kernels on the current CUDA device, synchronously.
 * Errors: SFFT4_EINVAL (out NULL, N not a power of two or out of range, K out of range,
 * l or q out of range, B1 invalid, delta not in (0, 1/2), window wider than N/2, or more
 * than 64 rounds in an iteration), SFFT4_ENOMEM, SFFT4_ECUDA.
 */
SFFT4_API int sfft4_plan(sfft4_plan_t* out, int64_t N, int64_t K, int32_t l, double q, uint64_t seed,
               const sfft4_opts* opts);

/* Releases a plan (NULL is ignored).  Synchronises the device first. */
SFFT4_API void sfft4_destroy(sfft4_plan_t plan);

/*
 * sfft4_execute -- one transform (signal index 0 of the Philox counter): the problem of
 * Section 2.1 (from the samples of x, the K largest coefficients X_f of its DFT, Eq. 1-2)
 * solved by the iterations of Section 3.1 -- per iteration the bucketization of Lemma 1
 * (random spectral permutation, Eq. 7-8; flat window, Eq. 9-10; fold and B-point DFT, Eq.
 * 11-13), the update by the coefficients found so far, the multiscale location of the large
 * buckets (Section 3.2, Eq. 15-19), the estimation of Eq. 14 and the merge x^m = x^{m-1} +
 * x'^m -- followed by the K-sparse output.
 *   x_dev      N complex64 samples (interleaved re, im float32), device memory, 8-byte aligned
 *   idx_dev    K int64 outputs: frequencies in [0, N) ascending; unused tail = -1
 *   val_dev    K complex128 outputs X_f in the Eq. 2 normalisation; unused tail = 0
 *   nfound_dev 1 int64 output: number of valid entries (<= K)
 *   votes_dev  K int8 outputs (levels that voted when the frequency was first accepted),
 *              may be NULL
 *   stream     cudaStream_t or NULL
 * Errors: SFFT4_EINVAL (NULL plan or output pointers), SFFT4_ECUDA (launch failure).
 */
SFFT4_API int sfft4_execute(sfft4_plan_t plan, const void* x_dev, int64_t* idx_dev, sfft4_c128* val_dev,
                  int64_t* nfound_dev, int8_t* votes_dev, void* stream);

/*
 * sfft4_execute_batched -- nsig independent instances of the problem of Section 2.1, each
 * solved by the iterations of Section 3.1 as in sfft4_execute, in one pass of batched
 * kernels (every kernel of an iteration covers all signals); signal i uses Philox counter
 * (i, m, 0, 0).
 *   nsig        1 <= nsig <= opts.max_batch of the plan
 *   x_dev       nsig * x_stride complex64 elements, device; signal i starts at
 *               x_dev + i * x_stride (x_stride >= N, in complex elements)
 *   idx_dev     nsig * K int64, val_dev nsig * K complex128, nfound_dev nsig int64,
 *   votes_dev   nsig * K int8 (may be NULL); row i belongs to signal i
 * Errors: SFFT4_EINVAL, SFFT4_ECUDA.
 */
SFFT4_API int sfft4_execute_batched(sfft4_plan_t plan, int32_t nsig, const void* x_dev, int64_t x_stride,
                          int64_t* idx_dev, sfft4_c128* val_dev, int64_t* nfound_dev,
                          int8_t* votes_dev, void* stream);

/*
 * sfft4_execute_batched_async -- sfft4_execute_batched (Section 2.1's problem for every
 * signal, by the iterations of Section 3.1) for a pipeline of batches: the transforms of
 * one batch (same arguments and results) run on the plan's own streams after
 * the work queued on `stream` so far, and `stream` does not wait for them, so consecutive
 * calls overlap (the decode chain of one batch with the gather of the next).  Calls use two
 * workspaces in turn; the first call allocates the second (a plan of the same transform and
 * options, created synchronously).  A third call queues behind the first one's work, so at
 * most two calls are in flight.
 *   Results are complete once sfft4_wait(plan, s) has been issued on a stream s and s has
 *   reached that point.  x_dev and the output buffers of a call must stay valid and
 *   unmodified until then; calls in flight together need distinct output buffers.
 *   A synchronous execute on the same plan waits for the asynchronous one that used the
 *   plan's own workspace.
 * Errors: SFFT4_EINVAL, SFFT4_ESTATE (a plan of sfft4_plan_batched, or opts.trace set),
 * SFFT4_ENOMEM, SFFT4_ECUDA.
 */
SFFT4_API int sfft4_execute_batched_async(sfft4_plan_t plan, int32_t nsig, const void* x_dev, int64_t x_stride,
                                          int64_t* idx_dev, sfft4_c128* val_dev, int64_t* nfound_dev,
                                          int8_t* votes_dev, void* stream);

/* Makes `stream` wait for every asynchronous execute issued so far on the plan.  Pipeline
 * control only: the paper has no counterpart.
 * Errors: SFFT4_EINVAL, SFFT4_ECUDA. */
SFFT4_API int sfft4_wait(sfft4_plan_t plan, void* stream);

/*
 * sfft4_execute_batched_host -- sfft4_execute_batched_async (Section 2.1's problem for every
 * signal, by the iterations of Section 3.1) on HOST buffers: the inputs are read from
 * page-locked host memory into the workspace's device copy by a kernel of the library
 * (zero-copy loads over the host link by 32 CTAs, which leave the other SMs to the
 * transforms of the batch before), the batch runs as an asynchronous execute, and the
 * results are copied back into the host outputs.  Consecutive calls overlap like
 * asynchronous executes (two workspaces in turn), so one batch's inputs cross the link while
 * the previous batch computes.
 *   x_host      nsig * x_stride complex64 elements in page-locked host memory (cudaHostAlloc,
 *               cudaMallocHost or cudaHostRegister; mapped, which unified addressing makes
 *               every page-locked allocation); signal i starts at x_host + i * x_stride
 *               (x_stride >= N).  16-byte aligned rows (even x_stride, 16-byte aligned
 *               x_host) are read 16 bytes at a time, others 8.
 *   idx_host, val_host, nfound_host, votes_host (may be NULL): as the device outputs of
 *               sfft4_execute_batched, in host memory; page-locked keeps the call
 *               asynchronous (pageable outputs are copied synchronously by the driver).
 *   Results are complete once sfft4_wait(plan, s) has been issued on a stream s and s has
 *   reached that point; x_host and the outputs of a call must stay valid and unmodified
 *   until then, and calls in flight together need distinct output buffers.
 *   The first host-buffer execute on each workspace allocates device copies of max_batch
 *   inputs and outputs (max_batch * N * 8 bytes, plus the outputs), kept until
 *   sfft4_destroy.
 * Errors: SFFT4_EINVAL (NULL pointers, sizes as sfft4_execute_batched, x_host not
 * page-locked host memory), SFFT4_ESTATE (a plan of sfft4_plan_batched, or opts.trace set),
 * SFFT4_ENOMEM, SFFT4_ECUDA.
 */
SFFT4_API int sfft4_execute_batched_host(sfft4_plan_t plan, int32_t nsig, const void* x_host, int64_t x_stride,
                                         int64_t* idx_host, sfft4_c128* val_host, int64_t* nfound_host,
                                         int8_t* votes_host, void* stream);

/*
 * sfft4_plan_batched -- plan of nsig transforms of different sizes, executed together
 * (batch of independent problems; each signal follows its own static schedule of Section 3.1).
 *   N[i], K[i]  size and sparsity of signal i, each within sfft4_plan's limits
 *   B1          NULL, or nsig first-iteration bucket counts (0 = the default of that signal;
 *               e.g. chosen per (N, K) by an autotuner); overrides opts->B1
 *   l, q, seed, opts  as for sfft4_plan, shared by every signal (opts.max_batch is ignored)
 * Signals with equal (N, K, B1) share one schedule; window tables are shared by (N, B).  Level m
 * of an execute runs iteration m of every signal that has one, as one fold launch, one or two
 * tensor-core DFT launches (one FP32 DFT launch per bucket count) and one decode launch per
 * round-count class, taking their work from job tables built here; the decode chain runs on
 * a second stream beside the bucketization of later levels.  Signal i uses Philox
 * counter (i, m, 0, 0), so it matches sfft4_plan(N[i], K[i], ...) run as signal i.
 * Errors: SFFT4_EINVAL (NULL pointers, nsig < 1, any size invalid), SFFT4_ENOMEM, SFFT4_ECUDA.
 */
SFFT4_API int sfft4_plan_batched(sfft4_plan_t* out, int32_t nsig, const int64_t* N, const int64_t* K,
                                 const int32_t* B1, int32_t l, double q, uint64_t seed, const sfft4_opts* opts);

/*
 * sfft4_execute_batched_v -- execute a plan from sfft4_plan_batched: for every signal i, the
 * problem of Section 2.1 for (N[i], K[i]) by the iterations of Section 3.1 on that signal's
 * own schedule (level m of the execute runs iteration m of every signal that has one).
 *   x_ptrs_dev  device array of nsig device pointers; signal i has N[i] complex64 samples
 *               (8-byte aligned) at x_ptrs_dev[i].  The array is read by the kernels, so its
 *               entries may change between executes (also under opts.graph)
 *   idx_dev     nsig * Kmax int64, val_dev nsig * Kmax complex128, votes_dev nsig * Kmax int8
 *               (may be NULL), nfound_dev nsig int64; row i (length Kmax = max K[i]) belongs
 *               to signal i, entries past its K[i] are -1 / 0
 * Errors: SFFT4_EINVAL (NULL pointers), SFFT4_ESTATE (plan not from sfft4_plan_batched),
 * SFFT4_ECUDA.
 */
SFFT4_API int sfft4_execute_batched_v(sfft4_plan_t plan, const void* const* x_ptrs_dev, int64_t* idx_dev,
                                      sfft4_c128* val_dev, int64_t* nfound_dev, int8_t* votes_dev,
                                      void* stream);

/*
 * sfft4_execute_batched_v_async -- sfft4_execute_batched_v (Section 2.1's problem per signal,
 * by the iterations of Section 3.1) as a pipeline of batches, with the
 * rules of sfft4_execute_batched_async, but with three workspaces in turn (the first call
 * makes the other two, plans of the same signals and options), so that the decode chains of
 * two batches overlap; at most three calls are in flight; results complete after sfft4_wait.  The pointer table, the
 * signals and the outputs of a call must stay valid and unmodified until then.
 * Errors: SFFT4_EINVAL, SFFT4_ESTATE (not a plan of sfft4_plan_batched), SFFT4_ENOMEM,
 * SFFT4_ECUDA.
 */
SFFT4_API int sfft4_execute_batched_v_async(sfft4_plan_t plan, const void* const* x_ptrs_dev, int64_t* idx_dev,
                                            sfft4_c128* val_dev, int64_t* nfound_dev, int8_t* votes_dev,
                                            void* stream);

typedef struct {
    int32_t nsig;
    int32_t n_classes;          /* distinct (N, K, B1) */
    int32_t n_levels;           /* longest schedule */
    int32_t kernels_per_execute;
    int64_t Kmax;               /* output row length */
    int64_t samples_per_execute;  /* distinct x positions read, summed over signals */
    int32_t precision;
} sfft4_batch_info;

#define SFFT4_MAX_VOTES 64
typedef struct {
    int64_t executes;            /* executes since the plan was made */
    int64_t transforms;          /* signals transformed since then */
    int64_t samples_per_execute; /* distinct x positions the last execute read (all signals) */
    int32_t iterations;          /* iterations (levels) of the longest schedule */
    int32_t kernels_per_execute; /* kernel launches of one execute */
    int32_t last_nsig;           /* signals of the last execute */
    int32_t reserved;
    int64_t last_found;          /* found-set entries after the last execute, all signals */
    int64_t votes_hist[SFFT4_MAX_VOTES + 1];  /* of those: how many were accepted with v votes */
} sfft4_run_stats;

/*
 * sfft4_stats -- counters of a plan (either kind) and the votes of the last execute's found
 * sets (levels that voted when each frequency was first accepted, Section 3.2).  Synchronises
 * the device.  Errors: SFFT4_EINVAL (NULL pointers), SFFT4_ECUDA.
 */
SFFT4_API int sfft4_stats(sfft4_plan_t plan, sfft4_run_stats* out);

/* Summary of a plan from sfft4_plan_batched.  Errors: SFFT4_EINVAL, SFFT4_ESTATE. */
SFFT4_API int sfft4_get_batch_info(sfft4_plan_t plan, sfft4_batch_info* info);

/* ----------------------------------------------------------------- introspection -- */
typedef struct {
    int64_t N, K;
    int32_t l, q_num;          /* q = q_num / 256 */
    int32_t B1, n_iters, max_R, precision;
    int64_t samples_per_transform;  /* distinct x positions read by one transform:
                                       sum over iterations of |union_s [tau_s-h, tau_s+h]| */
    int64_t found_capacity;    /* entries the found set of one signal can hold */
    int32_t kernels_per_execute;  /* kernel launches of one execute (any batch size) */
} sfft4_plan_info;

/* Static plan summary.  Errors: SFFT4_EINVAL on NULL arguments. */
SFFT4_API int sfft4_get_plan_info(sfft4_plan_t plan, sfft4_plan_info* info);

/*
 * sfft4_get_permutation -- the random spectral permutation of iteration m (1-based) of
 * signal `signal` (Section 2.2, Eq. 7-8): *sigma (odd) and *a in [0, N), drawn by
 * Philox4x64-10 with counter (signal, m, 0, 0) and key (seed, 0) as the kernels draw them.
 * The gather of round s reads x[(sigma t + a + sigma tau_s) mod N]; frequency f moves to
 * u = sigma f mod N.  Host-only; no device work.
 * Errors: SFFT4_EINVAL (NULL pointers, m out of range, signal < 0), SFFT4_ESTATE (plan from
 * sfft4_plan_batched).
 */
SFFT4_API int sfft4_get_permutation(sfft4_plan_t plan, int64_t signal, int32_t m, uint64_t* sigma, uint64_t* a);

#define SFFT4_MAX_ROUNDS 64
typedef struct {
    int32_t B;                 /* buckets B_m */
    int32_t S;                 /* multiscale levels; rounds R = S + 1 */
    int32_t n_c;               /* candidate buckets examined */
    int32_t h;                 /* window half-width (w = 2h + 1) */
    int64_t L;                 /* N / B_m */
    int64_t Lbar[SFFT4_MAX_ROUNDS];   /* nominal level lengths, levels 1..S (index 0..S-1) */
    int64_t tau[SFFT4_MAX_ROUNDS];    /* offsets tau_0 = 0 .. tau_S (index 0..S)           */
    uint32_t H[SFFT4_MAX_ROUNDS];     /* vote thresholds in 2^-32 turns, levels 1..S      */
    int64_t unique_samples;    /* |union_s [tau_s - h, tau_s + h]| */
} sfft4_iter_info;

/* Parameters of iteration m (1-based).  Errors: SFFT4_EINVAL (NULL or m out of range). */
SFFT4_API int sfft4_get_iter_info(sfft4_plan_t plan, int32_t m, sfft4_iter_info* info);

/*
 * sfft4_get_window -- copies the window of bucket count B used by the plan to host memory:
 * G (2h+1 float32 coefficients G_{-h..h}, as applied by the fold) and Ghat (3L/2 + 1
 * float32 values of the spectrum G'^_k, k = 0..3L/2).  Either output may be NULL.
 * Synchronous.  Errors: SFFT4_EINVAL (B not in the schedule), SFFT4_ECUDA.
 */
SFFT4_API int sfft4_get_window(sfft4_plan_t plan, int32_t B, float* G_host, float* Ghat_host);

/*
 * sfft4_bucketize -- frequency bucketization of one iteration alone (Lemma 1, Eq. 13):
 * for signal index `signal` and iteration m, writes the R x B raw bucket arrays
 * yhat_s[b] (complex64, row s = round s) to y_dev; no update, selection or location.
 * Errors: SFFT4_EINVAL, SFFT4_ECUDA.
 */
SFFT4_API int sfft4_bucketize(sfft4_plan_t plan, const void* x_dev, int32_t signal, int32_t m,
                    void* y_dev, void* stream);

/*
 * sfft4_trace_get -- after an execute on a plan made with opts.trace != 0, copies (to host,
 * synchronously) for iteration m of signal opts.trace_signal: the raw R x B bucket arrays (complex64,
 * y_host may be NULL) and the found set after the iteration: *nfound entries of
 * frequency (f_host, int64), value (v_host, complex128) and votes (votes_host, int8),
 * each of capacity `cap` entries (any of them may be NULL).
 * Errors: SFFT4_ESTATE (plan not traced or not executed), SFFT4_EINVAL, SFFT4_ECUDA.
 */
SFFT4_API int sfft4_trace_get(sfft4_plan_t plan, int32_t m, void* y_host, int64_t cap, int64_t* f_host,
                    sfft4_c128* v_host, int8_t* votes_host, int64_t* nfound);

/*
 * Kernel times of a profiled plan (opts.profile != 0), summed over the executes since the
 * last reset: per kernel kind (fold = permuted gather + window + fold, fft = B-point DFT,
 * decode = update/selection/location/estimation/merge, finalize) the number of launches
 * and their total duration from CUDA events recorded on the execution stream around each
 * launch; fold_samples counts the x samples the fold launches read (distinct positions per
 * signal and iteration, times the signals).  Synchronises with the events; reset != 0
 * clears the totals afterwards.
 * Errors: SFFT4_EINVAL (NULL), SFFT4_ESTATE (plan not made with opts.profile), SFFT4_ECUDA.
 */
typedef struct {
    int64_t fold_launches, fft_launches, decode_launches, finalize_launches;
    double fold_ms, fft_ms, decode_ms, finalize_ms;
    int64_t fold_samples;
} sfft4_profile;

SFFT4_API int sfft4_profile_get(sfft4_plan_t plan, sfft4_profile* out, int32_t reset);

/*
 * sfft4_gather_probe -- measures the device's throughput for the memory access pattern of
 * the gather (Lemma 1, step P0): independent random 8-byte loads, each CTA confined to one
 * signal of a batch.  Used as the achievable-bandwidth denominator of the gather's
 * roofline.  Reads x_dev (nsig signals of N complex64 at stride x_stride, N a power of two
 * <= 2^30); sink_dev is one float the kernel may write.  `blocks` CTAs of 512 threads each
 * issue iters x 4 loads; the timed launch follows one warm-up launch on `stream`.
 * Writes loads per second to *loads_per_second (host).  Synchronises with the stream.
 * Errors: SFFT4_EINVAL, SFFT4_ECUDA.
 */
SFFT4_API int sfft4_gather_probe(const void* x_dev, int32_t nsig, int64_t N, int64_t x_stride,
                                 float* sink_dev, int32_t blocks, int32_t iters,
                                 double* loads_per_second, void* stream);

/*
 * sfft4_gather_probe_ex -- sfft4_gather_probe with the knobs of a ceiling sweep: `threads` per
 * CTA (32..1024, a multiple of 32), `inflight` independent loads per thread at a time (4, 8 or
 * 16), and the L2 fetch granularity used during the measurement (l2_fetch_bytes 32, 64 or 128
 * bytes, restored afterwards; 0 = the context's current limit).  The footprint is nsig x N x 8
 * bytes: nsig = 1 keeps a 32 MB signal resident in L2, larger nsig exceed it.  The paper has
 * no counterpart (it measures the device, not the method).
 * Errors: SFFT4_EINVAL, SFFT4_ECUDA.
 */
SFFT4_API int sfft4_gather_probe_ex(const void* x_dev, int32_t nsig, int64_t N, int64_t x_stride,
                                    float* sink_dev, int32_t blocks, int32_t threads, int32_t iters,
                                    int32_t inflight, int32_t l2_fetch_bytes, double* loads_per_second,
                                    void* stream);

/*
 * sfft4_window_noalloc -- the flat window tables of sfft4_plan (G: 2h+1 float32
 * coefficients G_{-h..h}; Ghat: 3L/2+1 float32 values G'^_k, k = 0..3L/2, L = N/B) computed
 * into caller-provided device buffers without allocating any device memory.  The paper has
 * no counterpart: this entry point serves callers that cannot allocate device memory at the
 * point where they need the tables, because their memory is owned by another allocator (a
 * framework's caching allocator or a fixed pool) or because they cannot afford the implicit
 * device synchronisation of cudaMalloc/cudaFree.
 *   N, B, delta  as for sfft4_plan (N a power of two in [2^8, 2^30]; B a power of two in
 *                [16, min(4096, N/64)]; 0 < delta < 1/2)
 *   G_dev, Ghat_dev  device outputs with capacities G_cap >= 2h+1 and Ghat_cap >= 3L/2+1
 *                elements (h = ceil(B 4 sqrt2 erfcinv(delta) / (2 pi) * sqrt(2 ln(1/delta))))
 *   stream       cudaStream_t or NULL; the work is asynchronous on it
 * Its only scratch is one static device array of 131072 FP64 values (1 MiB, held by every GPU
 * that loads the library until the process exits), so windows longer than 131072
 * coefficients (B > 2048 at delta = 1e-8) are rejected with SFFT4_EINVAL.  The first call on
 * a device looks up that array's address (cudaGetSymbolAddress) once per device and CUDA
 * context (after the device's context is destroyed, e.g. by cudaDeviceReset, the next call
 * looks it up again); make that first call before any stream capture.  All calls share the array: calls that overlap on the GPU (on
 * different streams, or from different host threads) race and must be serialised by the
 * caller.
 * Errors: SFFT4_EINVAL (sizes, capacities, NULL outputs), SFFT4_ECUDA.
 */
SFFT4_API int sfft4_window_noalloc(int64_t N, int32_t B, double delta, float* G_dev, int64_t G_cap,
                                   float* Ghat_dev, int64_t Ghat_cap, void* stream);

/*
 * sfft4_sync_status -- synchronises the device and reports whether any bounded device-side
 * wait of this plan's kernels (the tensor-core DFT's wait for its accumulator) gave up since
 * the last call: SFFT4_ETIMEOUT if so (the affected outputs are incomplete), else SFFT4_OK.
 * Clears the flag.  Errors: SFFT4_EINVAL (NULL plan), SFFT4_ECUDA.
 */
SFFT4_API int sfft4_sync_status(sfft4_plan_t plan);

/*
 * sfft4_inject_status -- test hook: sets the plan's device status word to `value` (nonzero:
 * as a bounded device-side wait does when it gives up), synchronously, so that tests can
 * check sfft4_sync_status's reporting without making a device wait run out.  The paper has
 * no counterpart.  Errors: SFFT4_EINVAL (NULL plan), SFFT4_ECUDA.
 */
SFFT4_API int sfft4_inject_status(sfft4_plan_t plan, int32_t value);

/* Text of an error code (static storage). */
SFFT4_API const char* sfft4_strerror(int code);

/* Text of the last CUDA error seen by this thread inside the library (static storage). */
SFFT4_API const char* sfft4_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SFFT4_H */
