// Host planner of the sFFT4.0 library: validates parameters, builds the static schedule
// of iterations (Section 3.1, Lemma 2), the multiscale levels and offsets of each iteration
// (Section 3.2, Fig. 4), the fold segments, and allocates device tables and workspace.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "sfft4_internal.cuh"

using namespace sfft4;

namespace {

thread_local char g_cuda_err[256] = "no error";

int64_t pow2ceil(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

int ilog2(int64_t v) {
    int r = 0;
    while ((int64_t(1) << r) < v) ++r;
    return r;
}

// Nominal level lengths of a region of length L0 (Section 3.2): Lbar_{s+1} =
// ceil((q+1) Lbar_s / l) + 1 while Lbar_s > l and the length still shrinks.
std::vector<int64_t> levels(int64_t L0, int l, int qn) {
    std::vector<int64_t> out{L0};
    while (out.back() > l) {
        int64_t num = (int64_t)(kQDen + qn) * out.back();
        int64_t den = (int64_t)l * kQDen;
        int64_t nxt = (num + den - 1) / den + 1;
        if (nxt >= out.back()) break;
        out.push_back(nxt);
    }
    return out;
}

// Static schedule (B_m, K_m): K_1 = K, B_m = clamp(pow2ceil(ceil(beta K_m)), 16, B_1),
// K_{m+1} = K_m (1 - exp(-2 K_m / B_m)) until K_m < 1/2, then two more iterations.
std::vector<std::pair<int64_t, double>> schedule(int64_t K, int64_t B1, int max_iters) {
    std::vector<std::pair<int64_t, double>> out;
    double beta = (double)B1 / (double)K;
    double rem = (double)K;
    while ((int)out.size() < max_iters) {
        int64_t B = pow2ceil((int64_t)ceil(beta * rem));
        B = std::max<int64_t>(kBMin, std::min<int64_t>(B1, B));
        out.push_back({B, rem});
        rem = rem * (1.0 - exp(-2.0 * rem / (double)B));
        if (rem < 0.5) break;
    }
    for (int i = 0; i < 2; ++i)
        if ((int)out.size() < max_iters) out.push_back({out.back().first, rem});
    return out;
}

// Segments of the union of windows [tau_s - h, tau_s + h], s in [r0, r0 + nr).
void build_group(FoldGroup* g, const int64_t* tau, int r0, int nr, int64_t h) {
    g->r0 = r0;
    g->nr = nr;
    std::vector<std::pair<int64_t, int>> ev;  // (position, +/-(s+1))
    for (int s = r0; s < r0 + nr; ++s) {
        ev.push_back({tau[s] - h, s - r0 + 1});
        ev.push_back({tau[s] + h + 1, -(s - r0 + 1)});
    }
    std::sort(ev.begin(), ev.end());
    uint32_t mask = 0;
    g->nseg = 0;
    g->unique = 0;
    for (size_t i = 0; i < ev.size(); ++i) {
        int e = ev[i].second;
        if (e > 0) mask |= 1u << (e - 1);
        else mask &= ~(1u << (-e - 1));
        if (i + 1 < ev.size() && ev[i + 1].first > ev[i].first && mask) {
            g->t0[g->nseg] = ev[i].first;
            g->t1[g->nseg] = ev[i + 1].first;
            g->mask[g->nseg] = mask;
            g->unique += ev[i + 1].first - ev[i].first;
            g->nseg++;
        }
    }
}

void free_plan(sfft4_plan_s* p) {
    if (!p) return;
    if (p->owns_tables) {
        for (auto& w : p->wins) {
            cudaFree(w.G);
            cudaFree(w.Ghat);
            cudaFree(w.tw);
            cudaFree(w.dA1);
            cudaFree(w.dA2);
            cudaFree(w.tw4);
        }
    }
    void* bufs[] = {p->dec_iters, p->queue, p->iters_dev, p->z, p->zall, p->uall, p->y, p->u, p->status, p->F, p->ff, p->fv, p->fvotes, p->hkeys,
                    p->hvals, p->theta, p->fxexp, p->hx, p->hidx, p->hval, p->hnf, p->hvotes, p->trace_y, p->trace_F, p->trace_ff,
                    p->trace_fv, p->trace_votes};
    for (void* b : bufs) cudaFree(b);
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->gstream) cudaStreamDestroy(p->gstream);
    for (cudaEvent_t e : p->ev)
        if (e) cudaEventDestroy(e);
    if (p->dstream) cudaStreamDestroy(p->dstream);
    for (int s = 0; s < sfft4::kAsyncDepth; ++s) {
        if (p->ev_in[s]) cudaEventDestroy(p->ev_in[s]);
        if (p->ev_done[s]) cudaEventDestroy(p->ev_done[s]);
        if (p->astream[s]) cudaStreamDestroy(p->astream[s]);
    }
    if (p->ev_sync) cudaEventDestroy(p->ev_sync);
    for (cudaEvent_t e : p->ev_staged)
        if (e) cudaEventDestroy(e);
    if (p->hstream) cudaStreamDestroy(p->hstream);
    for (sfft4_plan_s* q : p->peer) free_plan(q);
    sfft4::destroy_group(p->grp);
    delete p;
}

}  // namespace

namespace sfft4 {

// Inverse complementary error function by Newton's method on erfc (0 < y < 1).
double erfcinv_newton(double y) {
    // start from the asymptotic form erfc(x) ~ exp(-x^2) / (x sqrt(pi)) for small y
    double x = (y < 0.5) ? sqrt(-log(y)) : 0.0;
    if (y >= 0.5) x = (1.0 - y) * 0.886226925452758;  // erfinv(z) ~ sqrt(pi)/2 z
    for (int i = 0; i < 100; ++i) {
        double f = erfc(x) - y;
        double d = -2.0 / sqrt(M_PI) * exp(-x * x);
        double step = f / d;
        x -= step;
        if (fabs(step) <= 1e-17 * fabs(x)) break;
    }
    return x;
}

// Window half-width: frequency box of half-width 3L/4 convolved with a Gaussian of std
// s_f = L / (4 sqrt 2 erfcinv(delta)); in time a Gaussian of std s_t = N / (2 pi s_f),
// truncated at delta: h = ceil(s_t sqrt(2 ln(1/delta))) (flat window of Eq. 9).
int64_t window_halfwidth(int64_t B, double delta, double* s_t_out) {
    double c = 4.0 * sqrt(2.0) * erfcinv_newton(delta);
    double s_t = (double)B * c / (2.0 * M_PI);
    if (s_t_out) *s_t_out = s_t;
    return (int64_t)ceil(s_t * sqrt(2.0 * log(1.0 / delta)));
}

int check_cuda(cudaError_t e) {
    if (e == cudaSuccess) return SFFT4_OK;
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SFFT4_ENOMEM : SFFT4_ECUDA;
}
}  // namespace sfft4

#define CK(call)                                   \
    do {                                           \
        int _rc = sfft4::check_cuda(call);         \
        if (_rc != SFFT4_OK) { free_plan(p); return _rc; } \
    } while (0)

extern "C" {

int sfft4_opts_default(sfft4_opts* o) {
    if (!o) return SFFT4_EINVAL;
    memset(o, 0, sizeof(*o));
    o->delta = 1e-8;
    o->precision = SFFT4_FP32;
    o->select_factor = 2.0;
    o->sig_floor = 1e-10;
    o->mag_tol = 0.5;
    o->max_iters = 64;
    o->max_batch = 1;
    return SFFT4_OK;
}

}  // extern "C"

namespace sfft4 {

// Kernel launches of one execute of a uniform plan: per iteration its fold groups, one FP32 DFT
// or one/two tensor-core DFT stages, one decode; one finalize.
int32_t uniform_kernels(const sfft4_plan_s* p, int nsig) {
    const bool sig_major = p->o.fold_order == SFFT4_FOLD_SIGNAL_MAJOR;
    const bool chain = decode_chain_used(p, nsig);
    // finalize, the fold launches covering every iteration (signal-major), the persistent decode
    int32_t k = 1 + (sig_major ? std::max<int32_t>(1, (int32_t)p->sm_fold.size()) : 0) + (chain ? 1 : 0);
    const bool tc = p->o.precision == SFFT4_BF16X3;
    int nsingle = 0, nfour = 0;  // BF16X3 DFT groups by stage count
    for (auto& ih : p->iters) {
        k += (sig_major ? 0 : (int32_t)ih.groups.size()) + (chain ? 0 : 1);  // folds, decode
        if (!(sig_major && tc)) k += (tc && ih.d.B > 64) ? 2 : 1;
        (ih.d.B > 64 ? nfour : nsingle)++;
    }
    // signal-major BF16X3: every iteration's DFT in grouped launches of up to 12 groups
    if (sig_major && tc) k += (nsingle + nfour + 11) / 12 + (nfour + 11) / 12;
    return k;
}

// Options with zero fields replaced by defaults, validated with the sizes (sfft4_plan's checks).
int plan_options(int64_t N, int64_t K, int32_t l, double q, const sfft4_opts* opts, sfft4_opts* out,
                 int* qn_out) {
    sfft4_opts o;
    sfft4_opts_default(&o);
    if (opts) {
        o = *opts;
        if (o.delta == 0) o.delta = 1e-8;
        if (o.select_factor == 0) o.select_factor = 2.0;
        if (o.sig_floor == 0) o.sig_floor = 1e-10;
        if (o.mag_tol == 0) o.mag_tol = 0.5;
        if (o.max_iters == 0) o.max_iters = 64;
        if (o.max_batch == 0) o.max_batch = 1;
    }
    if (N < 256 || (N & (N - 1)) || N > (int64_t(1) << 30)) return SFFT4_EINVAL;
    if (K < 1 || K > N / 64 || K > kKMax) return SFFT4_EINVAL;
    int qn = (int)floor(q * kQDen + 0.5);
    if (!(q >= 0) || l < 2 || l > 32 || (int64_t)l * kQDen <= kQDen + qn) return SFFT4_EINVAL;
    if (!(o.delta > 0 && o.delta < 0.5)) return SFFT4_EINVAL;
    if (o.precision != SFFT4_FP32 && o.precision != SFFT4_BF16X3) return SFFT4_EINVAL;
    if (o.max_batch < 1 || o.max_iters < 1 || o.max_iters > 256) return SFFT4_EINVAL;
    if (!(o.select_factor > 0) || !(o.mag_tol > 0) || o.min_votes < 0) return SFFT4_EINVAL;
    if (o.l2_fetch_bytes > 128) return SFFT4_EINVAL;
    if (o.location != SFFT4_LOC_MULTISCALE && o.location != SFFT4_LOC_TWO_ROUND) return SFFT4_EINVAL;
    if (o.fold_order != SFFT4_FOLD_SIGNAL_MAJOR && o.fold_order != SFFT4_FOLD_ITERATION_MAJOR) return SFFT4_EINVAL;
    if (o.decode_cluster < 0 || o.decode_cluster > 16 || (o.decode_cluster & (o.decode_cluster - 1))) return SFFT4_EINVAL;
    if (o.batch_exec != SFFT4_BATCH_PERSISTENT && o.batch_exec != SFFT4_BATCH_LEVELS) return SFFT4_EINVAL;
    if (o.fold_residues != 0 && o.fold_residues != 16 && o.fold_residues != 32 && o.fold_residues != 64)
        return SFFT4_EINVAL;
    if (o.fold_rounds < 0 || o.fold_rounds > kFoldRG) return SFFT4_EINVAL;
    // the two-round vote window is 1/(8N) turns: FP32 bucket arrays resolve it up to N = 2^20
    if (o.location == SFFT4_LOC_TWO_ROUND && N > (int64_t(1) << 20)) return SFFT4_EINVAL;
    int64_t B1 = o.B1;
    if (B1 == 0) {
        // two-round location tolerates few collisions: default 8 K buckets instead of 2 K
        const int64_t per = o.location == SFFT4_LOC_TWO_ROUND ? 8 : 2;
        B1 = std::max<int64_t>(kBMin, std::min<int64_t>({(int64_t)kBMax, N / 64, pow2ceil(per * K)}));
        // halve the default until the window of B1 buckets fits in N/2 (schedule of Section 3.1)
        while (B1 > kBMin && 2 * window_halfwidth(B1, o.delta, nullptr) + 1 > N / 2) B1 >>= 1;
    }
    if (B1 < kBMin || (B1 & (B1 - 1)) || B1 > N / 64 || B1 > kBMax) return SFFT4_EINVAL;
    o.B1 = (int32_t)B1;
    *out = o;
    *qn_out = qn;
    return SFFT4_OK;
}

// Host part of a plan: the static schedule of iterations (Section 3.1, reading R14), their
// levels, offsets, thresholds and location tables (Section 3.2), fold segments, and the list
// of bucket counts whose windows the plan needs.  No device work.
int plan_schedule(sfft4_plan_s* p) {
    const int64_t N = p->N, K = p->K;
    const int l = p->l, qn = p->qn;
    const sfft4_opts& o = p->o;
    auto sch = schedule(K, o.B1, o.max_iters);
    p->Fcap = 0;
    for (size_t i = 0; i < sch.size(); ++i) {
        int64_t B = sch[i].first;
        IterHost ih;
        memset(&ih.d, 0, sizeof(ih.d));
        IterDev& d = ih.d;
        d.m = (int32_t)i + 1;
        d.B = (int32_t)B;
        d.logB = ilog2(B);
        d.L = N / B;
        d.logL = ilog2(d.L);
        d.n_c = (int32_t)std::min<int64_t>(B, (int64_t)ceil(o.select_factor * std::max(sch[i].second, 1.0)));
        d.h = (int32_t)window_halfwidth(B, o.delta, nullptr);
        if (2 * (int64_t)d.h + 1 > N / 2) return SFFT4_EINVAL;
        // search region [bL - L, bL + L): pass band plus the transition bands (reading R5')
        if (o.location == SFFT4_LOC_TWO_ROUND) {
            // rounds tau = 0, 1: the 2L integers of the search region compete directly, phase
            // step 1/N; a lone tone's phase sits on an integer, so the vote takes 1/8 of it
            d.S = 1;
            d.R = 2;
            d.Lbar[0] = 2 * d.L;
            d.tau[0] = 0;
            d.tau[1] = 1;
            d.W[0] = (uint64_t)1 << (32 - p->n);
            d.H[0] = (uint32_t)(d.W[0] / 8);
            d.jscale[0] = (float)(1.0 / (double)d.W[0]);
        }
        std::vector<int64_t> lv = o.location == SFFT4_LOC_TWO_ROUND ? std::vector<int64_t>() : levels(2 * d.L, l, qn);
        int S = o.location == SFFT4_LOC_TWO_ROUND ? 1 : (int)lv.size();
        if (S + 1 > kMaxRounds) return SFFT4_EINVAL;
        d.S = S;
        d.R = S + 1;
        if (o.location != SFFT4_LOC_TWO_ROUND) d.tau[0] = 0;
        for (int s = 0; s < (int)lv.size(); ++s) {
            int64_t Lb = lv[s];
            d.Lbar[s] = Lb;
            int64_t ts;
            if (s < S - 1) {
                int64_t ext = ((int64_t)qn * Lb + (int64_t)l * kQDen - 1) / ((int64_t)l * kQDen);
                ts = N / (Lb + ext);
                d.H[s] = (uint32_t)((((int64_t)(kQDen + qn) * Lb * ts) << (32 - p->n)) /
                                    (2 * (int64_t)l * kQDen));
                d.W[s] = (uint64_t)(Lb * ts) << (32 - p->n);
                d.jscale[s] = (float)((double)l / (double)d.W[s]);
                for (int j = 0; j < l; ++j) {
                    d.Cj[s][j] = (uint32_t)(((uint64_t)(2 * j + 1) * d.W[s] + (uint64_t)l) / (uint64_t)(2 * l));
                    int64_t num = ((int64_t)2 * j * kQDen - qn) * Lb, den = (int64_t)2 * l * kQDen;
                    int64_t fq = num / den;
                    if (num % den != 0 && num < 0) --fq;
                    d.Dj[s][j] = (int32_t)fq;
                }
            } else {
                ts = N / Lb;
                d.H[s] = (uint32_t)((ts << (32 - p->n)) / 2);
                d.W[s] = (uint64_t)ts << (32 - p->n);
                d.jscale[s] = (float)(1.0 / (double)d.W[s]);
            }
            d.tau[s + 1] = ts;
        }
        // fold groups of up to kFoldRG rounds
        // residues per fold CTA: 64 (with 512 threads, 8 copies of each residue).  Measured
        // at 256 x (N = 2^22, K = 1000) on one GB300: 100.3 K transforms/s against 97.5 K with
        // 32 residues (16 copies); 128 residues were slower still.  Two warps' window
        // coefficient loads are 64 contiguous floats.
        ih.Wj = (int32_t)std::min<int64_t>(B, p->o.fold_residues ? p->o.fold_residues : 64);
        ih.unique = 0;
        // balanced groups of at most kFoldGroupMax rounds (the fold kernel's accumulator count
        // is the largest group of its launch)
        const int gmax = p->o.fold_rounds ? p->o.fold_rounds : kFoldGroupMax;
        const int ngr = (d.R + gmax - 1) / gmax, gsz = (d.R + ngr - 1) / ngr;
        for (int r0 = 0; r0 < d.R; r0 += gsz) {
            FoldGroup g;
            build_group(&g, d.tau, r0, std::min(gsz, d.R - r0), d.h);
            // P copies of each residue: every fold CTA has 512 threads (Wj residues x P), the
            // same in every job of a launch, so no thread of a launch sized by its largest job
            // idles.  Measured at 256 x (N = 2^22, K = 1000): 90.1 K transforms/s, against
            // 84.7 K with P sized for about 12 samples per thread (the B = 2048 tiles then
            // used 320 of the launch's 448 threads), 88.2 K with 384 and 75.4 K with 256
            // threads per tile.
            g.P = (int32_t)std::max<int64_t>(1, 512 / ih.Wj);
            ih.groups.push_back(g);
        }
        {
            FoldGroup all;
            // the union over all rounds (for the sample count) -- at most 2R segments
            std::vector<std::pair<int64_t, int64_t>> iv;
            for (int s = 0; s <= S; ++s) iv.push_back({d.tau[s] - d.h, d.tau[s] + d.h});
            std::sort(iv.begin(), iv.end());
            int64_t lo = iv[0].first, hi = iv[0].second, tot = 0;
            for (size_t k = 1; k < iv.size(); ++k) {
                if (iv[k].first > hi + 1) { tot += hi - lo + 1; lo = iv[k].first; hi = iv[k].second; }
                else hi = std::max(hi, iv[k].second);
            }
            tot += hi - lo + 1;
            ih.unique = std::min(tot, N);
            (void)all;
        }
        p->samples += ih.unique;
        // window of this bucket count
        int wi = -1;
        for (size_t k = 0; k < p->wins.size(); ++k)
            if (p->wins[k].B == B) wi = (int)k;
        if (wi < 0) {
            Window w;
            w.N = N;
            w.B = (int32_t)B;
            w.h = d.h;
            w.L = d.L;
            p->wins.push_back(w);
            wi = (int)p->wins.size() - 1;
        }
        ih.win = wi;
        p->Fcap += d.n_c;
        p->B_max = std::max<int32_t>(p->B_max, (int32_t)B);
        p->R_max = std::max<int32_t>(p->R_max, d.R);
        p->iters.push_back(ih);
    }
    p->Hlog = ilog2(2 * p->Fcap + 2);
    p->yoff.clear();
    p->ytot = 0;
    for (auto& ih : p->iters) {
        p->yoff.push_back(p->ytot);
        p->ytot += (int64_t)ih.d.R * ih.d.B;
    }
    return SFFT4_OK;
}

// Device tables of a plan: window G, G'^ and FFT twiddles per bucket count (and the split DFT
// matrices for BF16X3), then the iteration parameters.  With a cache, tables are shared by
// (N, B) with other plans of a batch and owned by the cache.
int plan_tables(sfft4_plan_s* p, std::vector<Window>* cache) {
    int rc = check_cuda(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device));
    if (rc) return rc;
    for (auto& w : p->wins) {
        if (cache) {
            bool hit = false;
            for (const Window& c : *cache)
                if (c.N == w.N && c.B == w.B) { w = c; hit = true; break; }
            if (hit) continue;
        }
        rc = build_window_tables(p, &w, p->o.delta);
        if (rc != SFFT4_OK) return rc;
        if (p->o.precision == SFFT4_BF16X3) {
            rc = check_cuda(cudaMalloc(&w.dA1, dft_tc_matrix_bytes()));
            if (!rc) rc = check_cuda(cudaMalloc(&w.dA2, dft_tc_matrix_bytes()));
            if (!rc) rc = check_cuda(cudaMalloc(&w.tw4, (size_t)w.B * sizeof(float2)));
            if (!rc) rc = build_dft_tc_tables(w.B, w.dA1, w.dA2, w.tw4);
            if (rc != SFFT4_OK) return rc;
        }
        if (cache) cache->push_back(w);
    }
    if (cache) p->owns_tables = false;
    for (auto& ih : p->iters) {
        const Window& w = p->wins[ih.win];
        ih.d.G = w.G;
        ih.d.Ghat = w.Ghat;
        ih.d.tw = w.tw;
    }
    size_t ni = p->iters.size();
    rc = check_cuda(cudaMalloc(&p->iters_dev, ni * sizeof(IterDev)));
    if (rc) return rc;
    std::vector<IterDev> hd(ni);
    for (size_t i = 0; i < ni; ++i) hd[i] = p->iters[i].d;
    return check_cuda(cudaMemcpy(p->iters_dev, hd.data(), ni * sizeof(IterDev), cudaMemcpyHostToDevice));
}

}  // namespace sfft4

extern "C" {

int sfft4_plan(sfft4_plan_t* out, int64_t N, int64_t K, int32_t l, double q, uint64_t seed,
               const sfft4_opts* opts) {
    if (!out) return SFFT4_EINVAL;
    *out = nullptr;
    sfft4_opts o;
    int qn = 0;
    int rc0 = plan_options(N, K, l, q, opts, &o, &qn);
    if (rc0) return rc0;
    // the iteration-major fold puts the signals of a batch in grid.y (at most 65535)
    if (o.fold_order == SFFT4_FOLD_ITERATION_MAJOR && o.max_batch > 65535) return SFFT4_EINVAL;
    if (o.trace && (o.trace_signal < 0 || o.trace_signal >= o.max_batch)) return SFFT4_EINVAL;
    sfft4_plan_s* p = new (std::nothrow) sfft4_plan_s();
    if (!p) return SFFT4_ENOMEM;
    p->N = N;
    p->n = ilog2(N);
    p->K = K;
    p->l = l;
    p->qn = qn;
    p->seed = seed;
    p->o = o;
    CK(cudaGetDevice(&p->device));
    if (o.l2_fetch_bytes >= 0) {
        // The gather reads 8-byte samples at random positions.  A 128-byte fetch per miss
        // moves up to 16x the needed DRAM bytes; 32 bytes (one sector) is the least, but the
        // iterations of a signal, folded together, draw neighbouring samples often enough
        // that 64-byte fetches come out ahead (measured at 256 x (N = 2^22, K = 1000): fold 1.97 ms
        // per execute with 64 B, 2.05 ms with 32 B, 2.57 ms with 128 B).
        // This is a limit of the calling process's CUDA context (a performance hint), not a
        // device setting.
        CK(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, o.l2_fetch_bytes ? o.l2_fetch_bytes : 64));
    }
    int rc = plan_schedule(p);
    if (!rc) rc = plan_tables(p, nullptr);
    if (rc) { free_plan(p); return rc; }
    const size_t ni = p->iters.size();
    size_t mb = (size_t)o.max_batch;
    size_t rb = (size_t)p->R_max * p->B_max;
    CK(cudaMalloc(&p->z, mb * rb * sizeof(float2)));
    CK(cudaMalloc(&p->y, mb * (size_t)p->ytot * sizeof(float2)));
    if (o.fold_order == SFFT4_FOLD_SIGNAL_MAJOR) {
        CK(cudaMalloc(&p->zall, mb * (size_t)p->ytot * sizeof(float2)));
        if (o.precision == SFFT4_BF16X3) CK(cudaMalloc(&p->uall, mb * (size_t)p->ytot * sizeof(float2)));
        const int rcs = sfft4::build_signal_major_fold(p);
        if (rcs) { free_plan(p); return rcs; }
    }
    CK(cudaStreamCreateWithFlags(&p->dstream, cudaStreamNonBlocking));
    p->ev.assign(ni + 2, nullptr);
    for (auto& e : p->ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaMalloc(&p->F, mb * sizeof(int32_t)));
    CK(cudaMalloc(&p->status, sizeof(int32_t)));
    CK(cudaMemset(p->status, 0, sizeof(int32_t)));
    if (o.precision == SFFT4_BF16X3) CK(cudaMalloc(&p->u, mb * rb * sizeof(float2)));
    CK(cudaMalloc(&p->ff, mb * p->Fcap * sizeof(int32_t)));
    CK(cudaMalloc(&p->fv, mb * p->Fcap * sizeof(double2)));
    CK(cudaMalloc(&p->fvotes, mb * p->Fcap * sizeof(int8_t)));
    CK(cudaMalloc(&p->hkeys, mb * ((size_t)1 << p->Hlog) * sizeof(int32_t)));
    CK(cudaMalloc(&p->hvals, mb * ((size_t)1 << p->Hlog) * sizeof(int32_t)));
    CK(cudaMalloc(&p->theta, mb * sizeof(float)));
    CK(cudaMalloc(&p->fxexp, mb * sizeof(int32_t)));
    if (o.fold_order == SFFT4_FOLD_SIGNAL_MAJOR && !o.trace) {
        const int rcd = sfft4::build_decode_chain(p);
        if (rcd) { free_plan(p); return rcd; }
    }
    if (o.trace) {
        CK(cudaMalloc(&p->trace_y, ni * rb * sizeof(float2)));
        CK(cudaMalloc(&p->trace_F, ni * sizeof(int32_t)));
        CK(cudaMalloc(&p->trace_ff, ni * p->Fcap * sizeof(int32_t)));
        CK(cudaMalloc(&p->trace_fv, ni * p->Fcap * sizeof(double2)));
        CK(cudaMalloc(&p->trace_votes, ni * p->Fcap * sizeof(int8_t)));
    }
    CK(cudaDeviceSynchronize());
    *out = p;
    return SFFT4_OK;
}

int sfft4_plan_batched(sfft4_plan_t* out, int32_t nsig, const int64_t* N, const int64_t* K, const int32_t* B1,
                       int32_t l, double q, uint64_t seed, const sfft4_opts* opts) {
    if (!out) return SFFT4_EINVAL;
    *out = nullptr;
    if (nsig < 1 || !N || !K) return SFFT4_EINVAL;
    // the batch's options, with its own default fold group size
    sfft4_opts ob;
    if (opts) ob = *opts;
    else sfft4_opts_default(&ob);
    if (ob.fold_rounds == 0) ob.fold_rounds = kFoldGroupMaxBatched;
    opts = &ob;
    sfft4_opts o;
    int qn = 0;
    for (int32_t i = 0; i < nsig; ++i) {
        sfft4_opts oi = ob;
        if (B1) oi.B1 = B1[i];
        int rc0 = plan_options(N[i], K[i], l, q, &oi, &o, &qn);
        if (rc0) return rc0;
    }
    sfft4_plan_s* p = new (std::nothrow) sfft4_plan_s();
    if (!p) return SFFT4_ENOMEM;
    p->l = l;
    p->qn = qn;
    p->seed = seed;
    p->o = o;
    p->o.trace = 0;
    CK(cudaGetDevice(&p->device));
    CK(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device));
    if (o.l2_fetch_bytes >= 0)
        CK(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, o.l2_fetch_bytes ? o.l2_fetch_bytes : 64));
    CK(cudaMalloc(&p->status, sizeof(int32_t)));
    CK(cudaMemset(p->status, 0, sizeof(int32_t)));
    int rc = build_group_plan(p, nsig, N, K, B1, l, q, seed, opts);
    if (rc) { free_plan(p); return rc; }
    p->bN.assign(N, N + nsig);
    p->bK.assign(K, K + nsig);
    if (B1) p->bB1.assign(B1, B1 + nsig);
    p->bq = q;
    p->bopts = ob;
    CK(cudaStreamCreateWithFlags(&p->dstream, cudaStreamNonBlocking));
    p->ev.assign(group_levels(p->grp) + 2, nullptr);
    for (auto& e : p->ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaDeviceSynchronize());
    *out = p;
    return SFFT4_OK;
}

void sfft4_destroy(sfft4_plan_t p) {
    if (!p) return;
    cudaDeviceSynchronize();
    free_plan(p);
}

int sfft4_get_plan_info(sfft4_plan_t p, sfft4_plan_info* info) {
    if (!p || !info) return SFFT4_EINVAL;
    if (p->grp) return SFFT4_ESTATE;
    memset(info, 0, sizeof(*info));
    info->N = p->N;
    info->K = p->K;
    info->l = p->l;
    info->q_num = p->qn;
    info->B1 = p->o.B1;
    info->n_iters = (int32_t)p->iters.size();
    info->max_R = p->R_max;
    info->precision = p->o.precision;
    info->samples_per_transform = p->samples;
    info->found_capacity = p->Fcap;
    info->kernels_per_execute = uniform_kernels(p, p->o.max_batch);
    return SFFT4_OK;
}

int sfft4_get_permutation(sfft4_plan_t p, int64_t signal, int32_t m, uint64_t* sigma, uint64_t* a) {
    if (p && p->grp) return SFFT4_ESTATE;
    if (!p || !sigma || !a || signal < 0 || m < 1 || m > (int32_t)p->iters.size()) return SFFT4_EINVAL;
    permutation_draw(p->seed, (uint64_t)signal, (uint64_t)p->iters[m - 1].d.m, (uint64_t)p->N, sigma, a);
    return SFFT4_OK;
}

int sfft4_get_iter_info(sfft4_plan_t p, int32_t m, sfft4_iter_info* info) {
    if (p && p->grp) return SFFT4_ESTATE;
    if (!p || !info || m < 1 || m > (int32_t)p->iters.size()) return SFFT4_EINVAL;
    const IterHost& ih = p->iters[m - 1];
    memset(info, 0, sizeof(*info));
    info->B = ih.d.B;
    info->S = ih.d.S;
    info->n_c = ih.d.n_c;
    info->h = ih.d.h;
    info->L = ih.d.L;
    for (int s = 0; s < ih.d.S; ++s) {
        info->Lbar[s] = ih.d.Lbar[s];
        info->H[s] = ih.d.H[s];
    }
    for (int s = 0; s <= ih.d.S; ++s) info->tau[s] = ih.d.tau[s];
    info->unique_samples = ih.unique;
    return SFFT4_OK;
}

int sfft4_get_window(sfft4_plan_t p, int32_t B, float* G_host, float* Ghat_host) {
    if (!p) return SFFT4_EINVAL;
    for (auto& w : p->wins) {
        if (w.B != B) continue;
        if (G_host) {
            int rc = check_cuda(cudaMemcpy(G_host, w.G, (2 * (size_t)w.h + 1) * sizeof(float),
                                           cudaMemcpyDeviceToHost));
            if (rc) return rc;
        }
        if (Ghat_host) {
            int rc = check_cuda(cudaMemcpy(Ghat_host, w.Ghat, (3 * (size_t)w.L / 2 + 1) * sizeof(float),
                                           cudaMemcpyDeviceToHost));
            if (rc) return rc;
        }
        return SFFT4_OK;
    }
    return SFFT4_EINVAL;
}

const char* sfft4_strerror(int code) {
    switch (code) {
        case SFFT4_OK: return "ok";
        case SFFT4_EINVAL: return "invalid argument";
        case SFFT4_ENOMEM: return "out of memory";
        case SFFT4_ECUDA: return "CUDA error";
        case SFFT4_ESTATE: return "invalid plan state";
        case SFFT4_ETIMEOUT: return "a bounded device wait gave up";
        default: return "unknown error";
    }
}

const char* sfft4_last_cuda_error(void) { return g_cuda_err; }

}  // extern "C"
