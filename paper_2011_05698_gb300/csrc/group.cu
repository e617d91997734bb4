// Batched sFFT4.0 over signals of different sizes N_i and sparsities K_i in one pass of
// table-driven kernels.
//
// Signals with equal (N, K, B1) share one static schedule ("class", Section 3.1); window
// tables are shared by (N, B).  The CTAs of every launch take their work from device tables
// built here: fold tiles (signal, iteration, fold group, residue slice), DFT columns grouped
// by bucket count, decode jobs (signal, iteration).  The bucketization of an iteration never
// reads the found sets, so it can run before the decode chain.  Two forms (opts.batch_exec):
//   persistent (default): all fold tiles in one launch (the tiles of a signal adjacent, so the
//     samples its iterations share are re-read from L2), all DFT columns in one or two
//     tensor-core launches (one per bucket count in FP32), then one decode launch of
//     persistent CTAs that take whole signals from a device queue, longest decode chains
//     first, and run each signal's iterations in order; four or five launches per execute;
//   levels: level m = iteration m of every signal that has one, its fold, DFT and decode
//     launches, the decode chain on a second stream overlapping later levels' bucketization.
// Both compute every tile, column and iteration identically, so their outputs are the same.
// A whole execute can be captured as one CUDA graph (opts.graph).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <tuple>

#include "sfft4_internal.cuh"

namespace sfft4 {

struct GroupLevel {
    struct Fold {
        int RG;
        int64_t off;
        int n, threads;
        size_t smem;
        int64_t samples;
    };
    struct Dft {
        int B;
        int64_t off;
        int n;
        Window w;
    };
    struct Dec {
        int rclass;
        int64_t off;
        int n;
        size_t smem;
    };
    std::vector<Fold> folds;
    std::vector<Dft> dfts;
    std::vector<Dec> decs;
};

struct Group {
    int nsig = 0;
    int64_t Kmax = 0;
    std::vector<sfft4_plan_s*> cls;    // one schedule per distinct (N, K)
    std::vector<int> slot_cls;
    std::vector<Window> wcache;        // tables shared by (N, B), owned here
    std::vector<GroupLevel> levels;
    // device tables
    FoldArgs* fold_jobs = nullptr;
    FoldTile* tiles = nullptr;
    const float2** zcols = nullptr;
    float2** ucols = nullptr;
    float2** ycols = nullptr;
    DecodeArgs* dec_jobs = nullptr;
    int32_t* dec_list = nullptr;
    FinalJob* fin_jobs = nullptr;
    // persistent form: every level's fold tiles in one list, DFT columns by bucket count over
    // all levels, per-signal decode chains (indices into dec_jobs) and the queue order
    GroupLevel::Fold all_fold{1, 0, 0, 0, 0, 0};
    FoldTile* all_tiles = nullptr;
    std::vector<GroupLevel::Dft> all_dfts;
    const float2** all_zcols = nullptr;
    float2** all_ucols = nullptr;
    float2** all_ycols = nullptr;
    int32_t* chain_off = nullptr;      // signal i's iterations: chain_args[chain_off[i] ..]
    int32_t* chain_len = nullptr;
    int32_t* chain_order = nullptr;
    int32_t* queue = nullptr;
    DecodeArgs* chain_args = nullptr;  // dec_jobs reordered signal by signal
    int chain_rclass = 0, chain_grid = 1;
    size_t chain_smem = 0;
    int kernels_persistent = 0;
    bool persistent = true;            // opts.batch_exec == SFFT4_BATCH_PERSISTENT
    // workspace
    void* arena = nullptr;
    int32_t* F = nullptr;
    int32_t* hkeys = nullptr;
    size_t hkeys_count = 0;
    int64_t samples = 0;
    int kernels = 0;
};

namespace {

void free_group(Group* g) {
    if (!g) return;
    for (sfft4_plan_s* c : g->cls) {
        cudaFree(c->iters_dev);
        delete c;
    }
    for (auto& w : g->wcache) {
        cudaFree(w.G);
        cudaFree(w.Ghat);
        cudaFree(w.tw);
        cudaFree(w.dA1);
        cudaFree(w.dA2);
        cudaFree(w.tw4);
    }
    void* bufs[] = {g->fold_jobs, g->tiles, g->zcols, g->ucols, g->ycols, g->dec_jobs,
                    g->dec_list, g->fin_jobs, g->arena, g->all_tiles, g->all_zcols, g->all_ucols,
                    g->all_ycols, g->chain_off, g->chain_len, g->chain_order, g->queue,
                    g->chain_args};
    for (void* b : bufs) cudaFree(b);
    delete g;
}

template <class T>
int upload(T** dst, const std::vector<T>& v) {
    if (v.empty()) return SFFT4_OK;
    int rc = check_cuda(cudaMalloc(dst, v.size() * sizeof(T)));
    if (rc) return rc;
    return check_cuda(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

void destroy_group(Group* g) { free_group(g); }

size_t group_levels(const Group* g) { return g->levels.size(); }

const FinalJob* group_final_jobs(const Group* g, int* nsig, int64_t* samples, int* kernels) {
    *nsig = g->nsig;
    *samples = g->samples;
    *kernels = g->persistent ? g->kernels_persistent : g->kernels;
    return g->fin_jobs;
}

int build_group_plan(sfft4_plan_s* p, int nsig, const int64_t* Ns, const int64_t* Ks, const int32_t* B1s,
                     int32_t l, double q, uint64_t seed, const sfft4_opts* opts) {
    Group* g = new (std::nothrow) Group();
    if (!g) return SFFT4_ENOMEM;
    p->grp = g;
    g->nsig = nsig;
    g->persistent = p->o.batch_exec == SFFT4_BATCH_PERSISTENT;
    // classes of equal (N, K, B1), each with its own static schedule
    std::map<std::tuple<int64_t, int64_t, int32_t>, int> cls_of;
    for (int i = 0; i < nsig; ++i) {
        sfft4_opts oi;
        if (opts) oi = *opts;
        else sfft4_opts_default(&oi);
        if (B1s) oi.B1 = B1s[i];
        auto key = std::make_tuple(Ns[i], Ks[i], oi.B1);
        auto itc = cls_of.find(key);
        if (itc == cls_of.end()) {
            sfft4_opts o;
            int qn = 0;
            int rc = plan_options(Ns[i], Ks[i], l, q, &oi, &o, &qn);
            if (rc) return rc;
            sfft4_plan_s* c = new (std::nothrow) sfft4_plan_s();
            if (!c) return SFFT4_ENOMEM;
            g->cls.push_back(c);
            c->N = Ns[i];
            c->n = 0;
            while ((int64_t(1) << c->n) < c->N) ++c->n;
            c->K = Ks[i];
            c->l = l;
            c->qn = qn;
            c->seed = seed;
            c->o = o;
            c->device = p->device;
            rc = plan_schedule(c);
            if (!rc) rc = plan_tables(c, &g->wcache);
            if (rc) return rc;
            itc = cls_of.emplace(key, (int)g->cls.size() - 1).first;
        }
        g->slot_cls.push_back(itc->second);
        g->Kmax = std::max<int64_t>(g->Kmax, Ks[i]);
    }
    // workspace arena: per signal z, y, (u), found set, hash; per-signal scalars
    struct Slot {
        size_t z, y, u, ff, fv, fvt, hk, hv;
    };
    std::vector<Slot> so(nsig);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t oF = take((size_t)nsig * 4), oTh = take((size_t)nsig * 4), oFx = take((size_t)nsig * 4);
    size_t hk_total = 0;
    for (int i = 0; i < nsig; ++i) hk_total += (size_t)1 << g->cls[g->slot_cls[i]]->Hlog;
    const size_t oHK = take(hk_total * 4);  // all hash keys contiguous (one reset memset)
    size_t hk_run = 0;
    for (int i = 0; i < nsig; ++i) {
        const sfft4_plan_s* c = g->cls[g->slot_cls[i]];
        // every iteration's folded arrays, four-step scratch (BF16X3) and bucket arrays, iteration
        // m at offset yoff[m] of each block, so that all folds may run before all DFTs
        const size_t yb = (size_t)c->ytot * sizeof(float2);
        so[i].z = take(yb);
        so[i].y = take(yb);
        so[i].u = (p->o.precision == SFFT4_BF16X3) ? take(yb) : 0;
        so[i].ff = take((size_t)c->Fcap * 4);
        so[i].fv = take((size_t)c->Fcap * 16);
        so[i].fvt = take((size_t)c->Fcap);
        so[i].hk = oHK + hk_run * 4;
        hk_run += (size_t)1 << c->Hlog;
        so[i].hv = take(((size_t)1 << c->Hlog) * 4);
    }
    int rc = check_cuda(cudaMalloc(&g->arena, off));
    if (rc) return rc;
    char* A = (char*)g->arena;
    g->F = (int32_t*)(A + oF);
    float* theta = (float*)(A + oTh);
    int32_t* fx = (int32_t*)(A + oFx);
    g->hkeys = (int32_t*)(A + oHK);
    g->hkeys_count = hk_total;

    // level tables
    int Mmax = 0;
    for (sfft4_plan_s* c : g->cls) Mmax = std::max<int>(Mmax, (int)c->iters.size());
    std::vector<FoldArgs> fjobs;
    std::vector<FoldTile> tiles;
    std::vector<const float2*> zc;
    std::vector<float2*> uc, yc;
    std::vector<DecodeArgs> djobs;
    std::vector<int32_t> dlist;
    // persistent form: per signal its fold jobs and decode jobs (iteration order), and the DFT
    // columns of every level by bucket count
    struct SigFoldJob {
        int job, nsl;
        int64_t per_tile;
    };
    std::vector<std::vector<SigFoldJob>> sig_fold(nsig);
    std::vector<std::vector<int>> sig_dec(nsig);
    std::map<int, std::vector<int64_t>> cols_by_B;   // indices into zc / uc / yc
    std::map<int, Window> win_by_B;
    for (int mi = 0; mi < Mmax; ++mi) {
        GroupLevel L;
        // fold tiles of every signal and fold group of the level in one launch, instantiated for
        // the level's largest rounds-per-group count (a group with fewer rounds leaves the extra
        // register accumulators unused; its arithmetic is unchanged)
        {
            GroupLevel::Fold f{1, (int64_t)tiles.size(), 0, 0, 0, 0};
            for (int i = 0; i < nsig; ++i) {
                const sfft4_plan_s* c = g->cls[g->slot_cls[i]];
                if (mi >= (int)c->iters.size()) continue;
                const IterHost& ih = c->iters[mi];
                for (const FoldGroup& fg : ih.groups) {
                    size_t smem = 0;
                    FoldArgs a = make_fold_args(c, mi, fg, &smem);
                    a.z = (float2*)(A + so[i].z) + c->yoff[mi];
                    a.signal0 = i;
                    const int job = (int)fjobs.size();
                    fjobs.push_back(a);
                    for (int sl = 0; sl < ih.d.B / ih.Wj; ++sl) tiles.push_back({job, sl});
                    const int nsl = ih.d.B / ih.Wj;
                    sig_fold[i].push_back({job, nsl, fg.unique / nsl});
                    g->all_fold.RG = std::max(g->all_fold.RG, (int)fg.nr);
                    g->all_fold.threads = std::max(g->all_fold.threads, ih.Wj * fg.P);
                    g->all_fold.samples += fg.unique;
                    f.RG = std::max(f.RG, (int)fg.nr);
                    f.threads = std::max(f.threads, ih.Wj * fg.P);
                    f.smem = std::max(f.smem, smem);
                    f.samples += fg.unique;
                }
            }
            f.n = (int)((int64_t)tiles.size() - f.off);
            f.smem = fold_smem(f.RG, f.threads);
            if (f.n > 0) L.folds.push_back(f);
        }
        // DFT columns by bucket count
        std::map<int, std::vector<int>> byB;
        for (int i = 0; i < nsig; ++i) {
            const sfft4_plan_s* c = g->cls[g->slot_cls[i]];
            if (mi < (int)c->iters.size()) byB[c->iters[mi].d.B].push_back(i);
        }
        for (auto& kv : byB) {
            GroupLevel::Dft d{kv.first, (int64_t)zc.size(), 0, Window()};
            for (int i : kv.second) {
                const sfft4_plan_s* c = g->cls[g->slot_cls[i]];
                const IterHost& ih = c->iters[mi];
                d.w = c->wins[ih.win];
                win_by_B[kv.first] = d.w;  // the DFT tables depend on B alone
                for (int r = 0; r < ih.d.R; ++r) {
                    cols_by_B[kv.first].push_back((int64_t)zc.size());
                    zc.push_back((const float2*)(A + so[i].z) + c->yoff[mi] + (int64_t)r * ih.d.B);
                    uc.push_back(so[i].u ? (float2*)(A + so[i].u) + c->yoff[mi] + (int64_t)r * ih.d.B : nullptr);
                    yc.push_back((float2*)(A + so[i].y) + c->yoff[mi] + (int64_t)r * ih.d.B);
                }
            }
            d.n = (int)((int64_t)zc.size() - d.off);
            L.dfts.push_back(d);
        }
        // decode jobs by round class
        for (int rcl = 0; rcl < 3; ++rcl) {
            GroupLevel::Dec d{rcl, (int64_t)dlist.size(), 0, 0};
            for (int i = 0; i < nsig; ++i) {
                const sfft4_plan_s* c = g->cls[g->slot_cls[i]];
                if (mi >= (int)c->iters.size()) continue;
                const IterDev& id = c->iters[mi].d;
                const int cl = id.R <= 8 ? 0 : (id.R <= 16 ? 1 : 2);
                if (cl != rcl) continue;
                DecodeArgs a = make_decode_args(c, mi);
                a.signal0 = i;
                a.y = (float2*)(A + so[i].y) + c->yoff[mi];
                a.F = g->F + i;
                a.ff = (int32_t*)(A + so[i].ff);
                a.fv = (double2*)(A + so[i].fv);
                a.fvotes = (int8_t*)(A + so[i].fvt);
                a.hkeys = (int32_t*)(A + so[i].hk);
                a.hvals = (int32_t*)(A + so[i].hv);
                a.theta = theta + i;
                a.fxexp = fx + i;
                dlist.push_back((int32_t)djobs.size());
                sig_dec[i].push_back((int)djobs.size());
                djobs.push_back(a);
                d.smem = std::max(d.smem, decode_smem_bytes(id.B));
                g->chain_rclass = std::max(g->chain_rclass, rcl);
                g->chain_smem = std::max(g->chain_smem, decode_smem_bytes(id.B));
            }
            d.n = (int)((int64_t)dlist.size() - d.off);
            if (d.n > 0) L.decs.push_back(d);
        }
        g->kernels += (int)(L.folds.size() + L.decs.size());
        if (p->o.precision == SFFT4_BF16X3) {
            std::vector<int> Bs;
            for (auto& d : L.dfts) Bs.push_back(d.B);
            g->kernels += dft_tc_launches(Bs.data(), (int)Bs.size());
        } else {
            g->kernels += (int)L.dfts.size();
        }
        g->levels.push_back(L);
    }
    g->kernels += 1;  // finalize

    // persistent form.  Fold tiles signal after signal (heaviest signals first), within a
    // signal its jobs heaviest tile first: the CTAs resident at a time gather from few signals.
    // The z arrays of one signal are reused by every iteration in the levels form (one R_max x
    // B_max block); here every iteration's fold must keep its own, at the offset of its bucket
    // arrays in y... so the persistent fold writes into the signal's y block and the DFT reads
    // from there: see the column tables below.
    {
        std::vector<int64_t> sig_samples(nsig, 0);
        for (int i = 0; i < nsig; ++i)
            for (const SigFoldJob& j : sig_fold[i]) sig_samples[i] += j.per_tile * j.nsl;
        std::vector<int> sorder(nsig);
        for (int i = 0; i < nsig; ++i) sorder[i] = i;
        std::stable_sort(sorder.begin(), sorder.end(), [&](int u, int v) { return sig_samples[u] > sig_samples[v]; });
        std::vector<FoldTile> at;
        for (int i : sorder) {
            std::vector<SigFoldJob> js = sig_fold[i];
            std::stable_sort(js.begin(), js.end(), [](const SigFoldJob& u, const SigFoldJob& v) { return u.per_tile > v.per_tile; });
            for (const SigFoldJob& j : js)
                for (int sl = 0; sl < j.nsl; ++sl) at.push_back({j.job, sl});
        }
        g->all_fold.n = (int)at.size();
        g->all_fold.smem = fold_smem(g->all_fold.RG, g->all_fold.threads);
        rc = upload(&g->all_tiles, at);
        if (rc) return rc;
    }
    // DFT columns of every level, by bucket count
    {
        std::vector<const float2*> azc;
        std::vector<float2*> auc, ayc;
        std::vector<int> Bs;
        for (auto& kv : cols_by_B) {
            GroupLevel::Dft d{kv.first, (int64_t)azc.size(), 0, win_by_B[kv.first]};
            for (int64_t ci : kv.second) {
                azc.push_back(zc[ci]);
                auc.push_back(uc[ci]);
                ayc.push_back(yc[ci]);
            }
            d.n = (int)((int64_t)azc.size() - d.off);
            g->all_dfts.push_back(d);
            Bs.push_back(kv.first);
        }
        rc = upload(&g->all_zcols, azc);
        if (!rc) rc = upload(&g->all_ucols, auc);
        if (!rc) rc = upload(&g->all_ycols, ayc);
        if (rc) return rc;
        g->kernels_persistent = 1 + (p->o.precision == SFFT4_BF16X3 ? dft_tc_launches(Bs.data(), (int)Bs.size())
                                                                     : (int)Bs.size()) + 1 + 1;
    }
    // decode chains: signal i's iterations in order, longest chains first
    {
        std::vector<DecodeArgs> cargs;
        std::vector<int32_t> coff(nsig), clen(nsig), corder(nsig);
        for (int i = 0; i < nsig; ++i) {
            coff[i] = (int32_t)cargs.size();
            clen[i] = (int32_t)sig_dec[i].size();
            for (int j : sig_dec[i]) cargs.push_back(djobs[j]);
            corder[i] = i;
        }
        std::stable_sort(corder.begin(), corder.end(), [&](int u, int v) { return clen[u] > clen[v]; });
        g->chain_grid = std::max(1, std::min(nsig, 2 * p->sm_count));
        rc = upload(&g->chain_args, cargs);
        if (!rc) rc = upload(&g->chain_off, coff);
        if (!rc) rc = upload(&g->chain_len, clen);
        if (!rc) rc = upload(&g->chain_order, corder);
        if (!rc) rc = check_cuda(cudaMalloc(&g->queue, sizeof(int32_t)));
        if (rc) return rc;
    }
    std::vector<FinalJob> fin(nsig);
    for (int i = 0; i < nsig; ++i) {
        const sfft4_plan_s* c = g->cls[g->slot_cls[i]];
        fin[i] = FinalJob{g->F + i, (const int32_t*)(A + so[i].ff), (const double2*)(A + so[i].fv),
                          (const int8_t*)(A + so[i].fvt), c->Fcap, c->K};
        g->samples += c->samples;
    }
    rc = upload(&g->fold_jobs, fjobs);
    if (!rc) rc = upload(&g->tiles, tiles);
    if (!rc) rc = upload(&g->zcols, zc);
    if (!rc) rc = upload(&g->ucols, uc);
    if (!rc) rc = upload(&g->ycols, yc);
    if (!rc) rc = upload(&g->dec_jobs, djobs);
    if (!rc) rc = upload(&g->dec_list, dlist);
    if (!rc) rc = upload(&g->fin_jobs, fin);
    return rc;
}

namespace {

// kernels launch_dft_tc_sets makes for these column sets (the profile counts each)
int dft_set_launches(const std::vector<DftColSet>& sets) {
    std::vector<int> Bs;
    for (const auto& c : sets) Bs.push_back(c.B);
    return dft_tc_launches(Bs.data(), (int)Bs.size());
}
struct GroupRun {
    const float2* const* x;
    int64_t* idx;
    sfft4_c128* val;
    int64_t* nfound;
    int8_t* votes;
};

// Persistent form: all fold tiles, all DFT columns, one persistent decode launch, finalize,
// in order on the caller's stream.
int group_body_persistent(sfft4_plan_s* p, const void* ctx, cudaStream_t st) {
    const GroupRun& r = *(const GroupRun*)ctx;
    Group* g = p->grp;
    int rc = check_cuda(cudaMemsetAsync(g->F, 0, (size_t)g->nsig * sizeof(int32_t), st));
    if (!rc) rc = check_cuda(cudaMemsetAsync(g->hkeys, 0xff, g->hkeys_count * sizeof(int32_t), st));
    if (!rc) rc = check_cuda(cudaMemsetAsync(g->queue, 0, sizeof(int32_t), st));
    if (rc) return rc;
    const GroupLevel::Fold& f = g->all_fold;
    cudaEvent_t ev = nullptr;
    rc = prof_begin(p, st, &ev);
    if (!rc) rc = launch_fold_multi(f.RG, g->fold_jobs, g->all_tiles, f.n, r.x, f.threads, f.smem, st);
    if (!rc) rc = prof_end(p, st, ev, kProfFold, f.samples);
    if (rc) return rc;
    if (p->o.precision == SFFT4_BF16X3) {
        std::vector<DftColSet> sets;
        for (const auto& d : g->all_dfts)
            sets.push_back(DftColSet{d.B, d.w.dA1, d.w.dA2, d.w.tw4, g->all_zcols + d.off, g->all_ucols + d.off,
                                     g->all_ycols + d.off, d.n});
        rc = prof_begin(p, st, &ev);
        if (!rc) rc = launch_dft_tc_sets(sets.data(), (int)sets.size(), p->status, p->sm_count, st);
        if (!rc) rc = prof_end(p, st, ev, kProfFft, 0, dft_set_launches(sets));
        if (rc) return rc;
    } else {
        for (const auto& d : g->all_dfts) {
            rc = prof_begin(p, st, &ev);
            if (!rc) rc = launch_fft_multi(g->all_zcols + d.off, g->all_ycols + d.off, d.n, d.B, d.w.tw, st);
            if (!rc) rc = prof_end(p, st, ev, kProfFft, 0);
            if (rc) return rc;
        }
    }
    rc = prof_begin(p, st, &ev);
    if (!rc) rc = launch_decode_chain(g->chain_rclass, g->chain_args, g->chain_off, g->chain_len, g->chain_order,
                                      g->nsig, g->queue, g->chain_grid, g->chain_smem, st);
    if (!rc) rc = prof_end(p, st, ev, kProfDecode, 0);
    if (!rc) rc = prof_begin(p, st, &ev);
    if (!rc) rc = launch_finalize_multi(g->fin_jobs, g->nsig, g->Kmax, r.idx, r.val, r.nfound, r.votes, st);
    if (!rc) rc = prof_end(p, st, ev, kProfFinalize, 0);
    return rc;
}

int group_body(sfft4_plan_s* p, const void* ctx, cudaStream_t st) {
    const GroupRun& r = *(const GroupRun*)ctx;
    Group* g = p->grp;
    if (g->persistent) return group_body_persistent(p, ctx, st);
    // bucketization of every level on the caller's stream, the decode chain on the plan's
    // decode stream (level m after its bucket arrays exist): the bucketization never reads
    // the found sets, so later levels' folds overlap earlier levels' decodes
    cudaStream_t ds = p->dstream;
    int rc = check_cuda(cudaMemsetAsync(g->F, 0, (size_t)g->nsig * sizeof(int32_t), st));
    if (!rc) rc = check_cuda(cudaMemsetAsync(g->hkeys, 0xff, g->hkeys_count * sizeof(int32_t), st));
    if (!rc) rc = check_cuda(cudaEventRecord(p->ev[0], st));
    if (!rc) rc = check_cuda(cudaStreamWaitEvent(ds, p->ev[0], 0));
    if (rc) return rc;
    for (size_t li = 0; li < g->levels.size(); ++li) {
        const GroupLevel& L = g->levels[li];
        for (const auto& f : L.folds) {
            cudaEvent_t ev = nullptr;
            rc = prof_begin(p, st, &ev);
            if (!rc) rc = launch_fold_multi(f.RG, g->fold_jobs, g->tiles + f.off, f.n, r.x, f.threads, f.smem, st);
            if (!rc) rc = prof_end(p, st, ev, kProfFold, f.samples);
            if (rc) return rc;
        }
        if (p->o.precision == SFFT4_BF16X3 && !L.dfts.empty()) {
            std::vector<DftColSet> sets;
            for (const auto& d : L.dfts)
                sets.push_back(DftColSet{d.B, d.w.dA1, d.w.dA2, d.w.tw4, g->zcols + d.off, g->ucols + d.off,
                                         g->ycols + d.off, d.n});
            cudaEvent_t ev = nullptr;
            rc = prof_begin(p, st, &ev);
            if (!rc) rc = launch_dft_tc_sets(sets.data(), (int)sets.size(), p->status, p->sm_count, st);
            if (!rc) rc = prof_end(p, st, ev, kProfFft, 0, dft_set_launches(sets));
            if (rc) return rc;
        } else {
            for (const auto& d : L.dfts) {
                cudaEvent_t ev = nullptr;
                rc = prof_begin(p, st, &ev);
                if (!rc) rc = launch_fft_multi(g->zcols + d.off, g->ycols + d.off, d.n, d.B, d.w.tw, st);
                if (!rc) rc = prof_end(p, st, ev, kProfFft, 0);
                if (rc) return rc;
            }
        }
        rc = check_cuda(cudaEventRecord(p->ev[1 + li], st));
        if (!rc) rc = check_cuda(cudaStreamWaitEvent(ds, p->ev[1 + li], 0));
        if (rc) return rc;
        for (const auto& d : L.decs) {
            cudaEvent_t ev = nullptr;
            rc = prof_begin(p, ds, &ev);
            if (!rc) rc = launch_decode_multi(d.rclass, g->dec_jobs, g->dec_list + d.off, d.n, d.smem, ds);
            if (!rc) rc = prof_end(p, ds, ev, kProfDecode, 0);
            if (rc) return rc;
        }
    }
    cudaEvent_t ev = nullptr;
    rc = prof_begin(p, ds, &ev);
    if (!rc) rc = launch_finalize_multi(g->fin_jobs, g->nsig, g->Kmax, r.idx, r.val, r.nfound, r.votes, ds);
    if (!rc) rc = prof_end(p, ds, ev, kProfFinalize, 0);
    if (!rc) rc = check_cuda(cudaEventRecord(p->ev[1 + g->levels.size()], ds));
    if (!rc) rc = check_cuda(cudaStreamWaitEvent(st, p->ev[1 + g->levels.size()], 0));
    return rc;
}
}  // namespace

}  // namespace sfft4

using namespace sfft4;

extern "C" {

int sfft4_execute_batched_v(sfft4_plan_t p, const void* const* x_ptrs_dev, int64_t* idx_dev,
                            sfft4_c128* val_dev, int64_t* nfound_dev, int8_t* votes_dev, void* stream) {
    if (!p || !x_ptrs_dev || !idx_dev || !val_dev || !nfound_dev) return SFFT4_EINVAL;
    if (!p->grp) return SFFT4_ESTATE;
    int rc0 = join_slot0(p, (cudaStream_t)stream);
    if (rc0) return rc0;
    const GroupRun r{(const float2* const*)x_ptrs_dev, idx_dev, val_dev, nfound_dev, votes_dev};
    const uint64_t key[8] = {2, (uint64_t)(uintptr_t)x_ptrs_dev, (uint64_t)(uintptr_t)idx_dev,
                             (uint64_t)(uintptr_t)val_dev, (uint64_t)(uintptr_t)nfound_dev,
                             (uint64_t)(uintptr_t)votes_dev, 0, 0};
    int rc = graph_run(p, key, (cudaStream_t)stream, group_body, &r);
    if (!rc) rc = mark_sync(p, (cudaStream_t)stream);
    if (!rc) {
        p->executed = true;
        ++p->n_executes;
        p->n_transforms += p->grp->nsig;
        p->last_nsig = p->grp->nsig;
    }
    return rc;
}

int sfft4_execute_batched_v_async(sfft4_plan_t p, const void* const* x_ptrs_dev, int64_t* idx_dev,
                                  sfft4_c128* val_dev, int64_t* nfound_dev, int8_t* votes_dev, void* stream) {
    if (!p || !x_ptrs_dev || !idx_dev || !val_dev || !nfound_dev) return SFFT4_EINVAL;
    if (!p->grp) return SFFT4_ESTATE;
    sfft4_plan_s* w = nullptr;
    cudaStream_t as = nullptr;
    int rc = async_begin(p, (cudaStream_t)stream, &w, &as);
    if (!rc) rc = sfft4_execute_batched_v(w, x_ptrs_dev, idx_dev, val_dev, nfound_dev, votes_dev, as);
    if (!rc) rc = async_end(p, as);
    return rc;
}

int sfft4_get_batch_info(sfft4_plan_t p, sfft4_batch_info* info) {
    if (!p || !info) return SFFT4_EINVAL;
    if (!p->grp) return SFFT4_ESTATE;
    const Group* g = p->grp;
    memset(info, 0, sizeof(*info));
    info->nsig = g->nsig;
    info->n_classes = (int32_t)g->cls.size();
    info->n_levels = (int32_t)g->levels.size();
    info->kernels_per_execute = g->persistent ? g->kernels_persistent : g->kernels;
    info->Kmax = g->Kmax;
    info->samples_per_execute = g->samples;
    info->precision = p->o.precision;
    return SFFT4_OK;
}

}  // extern "C"
