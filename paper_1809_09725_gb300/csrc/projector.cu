// projector.cu -- precision dispatch and C entry points of the dynamic
// projector pair (Sec. 4, Eqs. radapr and radadjapr).  The kernels live in
// projector_impl.cuh and are instantiated per precision in projector_*.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "projector_impl.cuh"
#include "fold_impl.cuh"

namespace dr {

dr_status ensure_fold_scratch(dr_plan *P) {
    if (P->d_gt) return DR_OK;
    cudaError_t e = cudaMalloc(&P->d_gt, std::max<size_t>(P->gt_bytes, 16));
    if (e != cudaSuccess) {
        P->d_gt = nullptr;
        return cuda_fail(e, "folded-data scratch allocation");
    }
    return DR_OK;
}

dr_status ensure_split_scratch(dr_plan *P, size_t bytes) {
    if (P->d_ru_split && P->ru_split_bytes >= bytes) return DR_OK;
    if (P->d_ru_split) {
        cudaError_t e = cudaFree(P->d_ru_split);
        P->d_ru_split = nullptr;
        P->ru_split_bytes = 0;
        if (e != cudaSuccess) return cuda_fail(e, "split scratch release");
    }
    cudaError_t e = cudaMalloc(&P->d_ru_split, bytes);
    if (e != cudaSuccess) {
        P->d_ru_split = nullptr;
        return cuda_fail(e, "split scratch allocation");
    }
    P->ru_split_bytes = bytes;
    return DR_OK;
}

// variant 0: direct (every projection at its own angle); 1: half-turn fold.
// calc: buffers are compute typed (float for F32/BF16 plans, double for F64).
dr_status launch_fwd_variant(dr_plan *P, int variant, bool calc, const void *u, void *out, const void *gm,
                             int mode, double sigma, cudaStream_t st) {
    if (variant == 1 && P->fold_U > 0 && P->fold_fwd_ok) {
        if (P->prec == DR_BF16_F32ACC && !calc) return FoldOps<bf16, float>::fwd(P, u, out, gm, mode, sigma, st);
        return FoldOps<float, float>::fwd(P, u, out, gm, mode, sigma, st);
    }
    if (variant == 2 && P->fold_U > 0 && P->fold2_ok) {
        if (P->prec == DR_BF16_F32ACC && !calc) return FoldOps<bf16, float>::fwd2(P, u, out, gm, mode, sigma, st);
        return FoldOps<float, float>::fwd2(P, u, out, gm, mode, sigma, st);
    }
    switch (P->prec) {
        case DR_F32: return ProjOps<float, float>::fwd(P, u, out, gm, mode, sigma, st);
        case DR_BF16_F32ACC:
            if (calc) return ProjOps<float, float>::fwd(P, u, out, gm, mode, sigma, st);
            return ProjOps<bf16, float>::fwd(P, u, out, gm, mode, sigma, st);
        case DR_F64: return ProjOps<double, double>::fwd(P, u, out, gm, mode, sigma, st);
    }
    return fail(DR_EINVAL, "bad precision");
}

dr_status launch_adj_variant(dr_plan *P, int variant, bool calc, const void *g, void *u, double alpha,
                             double beta, bool u_calc, cudaStream_t st) {
    if (variant == 1 && P->fold_U > 0) {
        dr_status s = ensure_fold_scratch(P);
        if (s != DR_OK) return s;
        if (P->prec == DR_BF16_F32ACC && !calc)
            return FoldOps<bf16, float>::adj(P, g, u, alpha, beta, u_calc, st);
        return FoldOps<float, float>::adj(P, g, u, alpha, beta, u_calc, st);
    }
    switch (P->prec) {
        case DR_F32: return ProjOps<float, float>::adj(P, g, u, alpha, beta, u_calc, st);
        case DR_BF16_F32ACC:
            if (calc) return ProjOps<float, float>::adj(P, g, u, alpha, beta, u_calc, st);
            return ProjOps<bf16, float>::adj(P, g, u, alpha, beta, u_calc, st);
        case DR_F64: return ProjOps<double, double>::adj(P, g, u, alpha, beta, u_calc, st);
    }
    return fail(DR_EINVAL, "bad precision");
}

static int fwd_choice(const dr_plan *P) { return P->var_fwd >= 0 ? P->var_fwd : P->sel_fwd; }
// storage-typed calls on BF16 plans run the bf16-strip kernels, timed separately
static int fwd_choice_st(const dr_plan *P) {
    return P->var_fwd >= 0 ? P->var_fwd : (P->prec == DR_BF16_F32ACC ? P->sel_fwd_st : P->sel_fwd);
}
static int adj_choice(const dr_plan *P) { return P->var_adj >= 0 ? P->var_adj : P->sel_adj; }

dr_status launch_fwd(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                     cudaStream_t st) {
    return launch_fwd_variant(P, fwd_choice_st(P), false, u, out, gm, mode, sigma, st);
}

dr_status launch_adj(dr_plan *P, const void *g, void *u, double alpha, double beta, bool u_calc,
                     cudaStream_t st) {
    return launch_adj_variant(P, adj_choice(P), false, g, u, alpha, beta, u_calc, st);
}

// Compute-typed variants for the solvers: all buffers are float (F32 and
// BF16 plans) or double (F64 plans).
dr_status launch_fwd_calc(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                          cudaStream_t st) {
    return launch_fwd_variant(P, fwd_choice(P), true, u, out, gm, mode, sigma, st);
}

dr_status launch_adj_calc(dr_plan *P, const void *g, void *u, double alpha, double beta, cudaStream_t st) {
    return launch_adj_variant(P, adj_choice(P), true, g, u, alpha, beta, true, st);
}

// y = R*R x: with the two-kernel folded forward and the folded adjoint, the
// static transforms are mixed per distinct angle and back-projected directly;
// otherwise forward into gscratch, then adjoint.
dr_status launch_normal_calc(dr_plan *P, const void *x, void *y, void *gscratch, cudaStream_t st) {
    if (P->prec != DR_F64 && P->fold_U > 0 && P->fold2_ok && P->d_fold_gram && fwd_choice(P) == 2 &&
        adj_choice(P) == 1)
        return FoldOps<float, float>::normal(P, x, y, st);
    dr_status s = launch_fwd_calc(P, x, gscratch, nullptr, 0, 0.0, st);
    if (s != DR_OK) return s;
    return launch_adj_calc(P, gscratch, y, 1.0, 0.0, st);
}

// Autotuner: time the direct and folded variants of both projectors on the
// plan's own geometry (compute-typed scratch buffers supplied by the
// caller, contents overwritten) and keep the faster of each.  Explicit
// choices made with dr_plan_set_variant are left alone.
// Process-wide cache of autotuner decisions, keyed by everything that
// defines the operators (sizes, basis, precision, and the acquisition
// angles and times), so every plan of the same problem runs the same
// kernels and produces bit-identical results.
struct TuneKey {
    int nx, ny, nz, ns, K, m, nt, basis, prec;
    uint64_t hash;
    bool operator<(const TuneKey &o) const {
        return std::tie(nx, ny, nz, ns, K, m, nt, basis, prec, hash) <
               std::tie(o.nx, o.ny, o.nz, o.ns, o.K, o.m, o.nt, o.basis, o.prec, o.hash);
    }
};
struct TuneVal {
    int fwd, adj, lines, async, lines_st, async_st, f2_gi, f2_lines, f2_lines_st, fwd_st, f2_split, f2_async,
        f2_async_st, adj_pp, f2_bv, f2_gi_st;
    double ms[5];
};
static std::mutex g_tune_mutex;
static std::map<TuneKey, TuneVal> g_tune_cache;

static TuneKey tune_key(const dr_plan *P) {
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the bytes of theta and t
    auto mix = [&h](const std::vector<double> &v) {
        const unsigned char *b = reinterpret_cast<const unsigned char *>(v.data());
        for (size_t i = 0; i < v.size() * sizeof(double); ++i) h = (h ^ b[i]) * 1099511628211ull;
    };
    mix(P->theta);
    mix(P->t);
    return TuneKey{P->nx, P->ny, P->nz, P->ns, P->K, P->m, P->nt, (int)P->basis, (int)P->prec, h};
}

dr_status autotune(dr_plan *P, void *u_scratch, void *g_scratch) {
    if (P->fold_U == 0) {
        P->tuned = true;
        return DR_OK;
    }
    const TuneKey key = tune_key(P);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            P->sel_fwd = it->second.fwd;
            P->sel_adj = it->second.adj;
            P->fold_lines = it->second.lines;
            P->fold_async = it->second.async;
            P->fold_lines_st = it->second.lines_st;
            P->fold_async_st = it->second.async_st;
            P->fold2_gi = it->second.f2_gi;
            P->fold2_gi_st = it->second.f2_gi_st;
            P->fold2_lines = it->second.f2_lines;
            P->fold2_lines_st = it->second.f2_lines_st;
            P->sel_fwd_st = it->second.fwd_st;
            P->fold2_split = P->split_off ? 1 : it->second.f2_split;
            P->fold2_async = it->second.f2_async;
            P->fold2_async_st = it->second.f2_async_st;
            P->fold_adj_pp = it->second.adj_pp;
            P->fold2_bv = it->second.f2_bv;
            for (int i = 0; i < 5; ++i) P->tune_ms[i] = it->second.ms[i];
            P->tuned = true;
            return DR_OK;
        }
    }
    cudaStream_t st = P->graph_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    struct EventPair {  // released on every return path
        cudaEvent_t *a, *b;
        ~EventPair() {
            if (*a) cudaEventDestroy(*a);
            if (*b) cudaEventDestroy(*b);
        }
    } events_guard{&e0, &e1};
    DR_CUDA_TRY(cudaEventCreate(&e0));
    DR_CUDA_TRY(cudaEventCreate(&e1));
    const size_t cs = calc_size(P->prec);
    DR_CUDA_TRY(cudaMemsetAsync(u_scratch, 0, nu_elems(P) * cs, st));
    DR_CUDA_TRY(cudaMemsetAsync(g_scratch, 0, ng_elems(P) * cs, st));
    double ms[5] = {1e30, 1e30, 1e30, 1e30, 1e30};
    double ms_st1 = 1e30, ms_st2 = 1e30;  // bf16-strip kernels of BF16 plans: fold, fold in two kernels
    // launches per trial: one warm-up, then the timed ones (reps - 1; the
    // screening trials and the direct variant, timed only for comparison, take one)
    // a serving job canceled while its plan is being tuned stops between trials
    auto canceled = [&]() { return P->cancel && P->cancel->load(std::memory_order_relaxed); };
    auto time_fwd = [&](int v, double &best, bool calc = true, int reps = 3) -> dr_status {
        if (canceled()) return fail(DR_ECANCELED, "autotune: canceled");
        for (int rep = 0; rep < reps; ++rep) {
            DR_CUDA_TRY(cudaEventRecord(e0, st));
            dr_status s = launch_fwd_variant(P, v, calc, u_scratch, g_scratch, nullptr, 0, 0.0, st);
            if (s != DR_OK) return s;
            DR_CUDA_TRY(cudaEventRecord(e1, st));
            DR_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.f;
            DR_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            if (rep > 0) best = std::min(best, (double)t);
        }
        return DR_OK;
    };
    // Strip-height search: the heights 2, 4, 8, 16 (those within rmax, and the
    // largest that fits), then the neighbours of the best one among
    // 1, 2, 3, 4, 6, 8, 12, 16.  run(lines, t) times one configuration; best_t
    // may come in holding another configuration's time, and `improved` says
    // whether one of these heights beat it.
    auto search_lines = [&](int rmax, auto run, int &best_lines, double &best_t, bool &improved) -> dr_status {
        const int all[] = {1, 2, 3, 4, 6, 8, 12, 16};
        bool tried[8] = {};
        improved = false;
        int best_i = -1;
        auto try_one = [&](int i) -> dr_status {
            if (i < 0 || i > 7 || tried[i] || all[i] > rmax) return DR_OK;
            tried[i] = true;
            double t = 1e30;
            dr_status s = run(all[i], t);
            if (s != DR_OK) return s;
            if (t < best_t) {
                best_t = t;
                best_lines = all[i];
                best_i = i;
                improved = true;
            }
            return DR_OK;
        };
        int imax = 0;
        while (imax < 7 && all[imax + 1] <= rmax) ++imax;
        for (int i : {1, 3, 5, 7, imax}) {
            dr_status s = try_one(i);
            if (s != DR_OK) return s;
        }
        if (!tried[1]) {  // rmax < 2
            dr_status s = try_one(0);
            if (s != DR_OK) return s;
        }
        if (best_i >= 0) {
            const int bi = best_i;
            for (int i : {bi - 1, bi + 1}) {
                dr_status s = try_one(i);
                if (s != DR_OK) return s;
            }
        }
        return DR_OK;
    };
    {
        dr_status s = time_fwd(0, ms[0], true, 2);
        if (s != DR_OK) return s;
    }
    if (P->fold_fwd_ok) {
        // folded forward: strip lines per buffer and staging mode
        // (every choice marches each ray over the same lines in the same order,
        // so the result does not depend on it)
        int best_lines = P->fold_R, best_async = 0;
        const int async_ok = P->m == P->M && ((P->prec == DR_F32 && P->M % 4 == 0) ||
                                              (P->prec == DR_BF16_F32ACC && P->M % 8 == 0));
        for (int as = 0; as <= async_ok; ++as) {
            // both buffers of the double-buffered mode share the strip budget
            P->fold_async = as;
            bool better = false;
            dr_status s = search_lines(
                as ? P->fold_R / 2 : P->fold_R,
                [&](int lines, double &t) {
                    P->fold_lines = lines;
                    // with the two-kernel form available, the fused kernel is timed
                    // for comparison only (one timed launch per trial)
                    return time_fwd(1, t, true, P->fold2_ok ? 2 : 3);
                },
                best_lines, ms[1], better);
            if (s != DR_OK) return s;
            if (better) best_async = as;
        }
        P->fold_lines = best_lines;
        P->fold_async = best_async;
        if (P->prec == DR_BF16_F32ACC) {
            // the storage-typed (bf16 strip) kernel of the operator calls: its own choice
            // (the scratch buffers are float sized, large enough for bf16 data)
            const int async_st_ok = P->m == P->M && P->M % 8 == 0;
            double best_t = 1e30;
            int bl = P->fold_R, ba = 0;
            for (int as = 0; as <= async_st_ok; ++as) {
                P->fold_async_st = as;
                bool better = false;
                dr_status s = search_lines(
                    as ? P->fold_R / 2 : P->fold_R,
                    [&](int lines, double &t) {
                        P->fold_lines_st = lines;
                        return time_fwd(1, t, false);
                    },
                    bl, best_t, better);
                if (s != DR_OK) return s;
                if (better) ba = as;
            }
            P->fold_lines_st = bl;
            P->fold_async_st = ba;
            ms_st1 = best_t;
        }
    }
    if (P->fold2_ok) {
        // two-kernel folded forward: coefficient group and CTA size, strip
        // height, staging mode, line chunks.  Group, CTA size, strip height and
        // staging change only which CTA computes a ray sum and when its lines
        // are copied: results do not depend on them.
        auto run2 = [&](bool calc, int reps = 3) {
            return [&, calc, reps](int lines, double &t) {
                if (calc) P->fold2_lines = lines;
                else P->fold2_lines_st = lines;
                return time_fwd(2, t, calc, reps);
            };
        };
        bool better = false;
        int bgi = P->fold2_gi, bl = P->fold2_lines;
        P->fold2_split = 1;
        P->fold2_async = 0;
        P->fold2_bv = 0;
        // screen the group / CTA configurations, each with synchronous and
        // double-buffered cp.async strips (twice the strip memory, so possibly
        // fewer CTAs per SM) at two strip heights; refine the two best, then
        // try triple buffering on the best
        auto gi_ok = [&](int gi) {
            const int MC = fold_static_mc(gi);
            return P->fold2_R[gi] >= 1 && !(MC == 8 && P->m <= 4) &&
                   (size_t)P->nz * ((P->m + MC - 1) / MC) <= 65535;
        };
        struct Cand {
            double t;
            int gi, async, lines;
        };
        std::vector<Cand> cands;
        for (int gi = 0; gi < kFold2Configs; ++gi) {
            if (!gi_ok(gi)) continue;
            P->fold2_gi = gi;
            for (int as = 0; as < 2; ++as) {
                P->fold2_async = as;
                Cand best{1e30, gi, as, 1};
                for (int c : {4, std::min(12, P->fold2_R[gi])}) {
                    if (c > P->fold2_R[gi] || (c == best.lines && best.t < 1e30)) continue;
                    double t = 1e30;
                    dr_status s = run2(true, 2)(c, t);
                    if (s != DR_OK) return s;
                    if (t < best.t) best = Cand{t, gi, as, c};
                }
                if (best.t < 1e30) cands.push_back(best);
            }
        }
        std::sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) { return a.t < b.t; });
        int basync = 0;
        for (size_t i = 0; i < cands.size() && i < 2; ++i) {
            P->fold2_gi = cands[i].gi;
            P->fold2_async = cands[i].async;
            int l2 = cands[i].lines;
            if (cands[i].t < ms[4]) {
                ms[4] = cands[i].t;
                bgi = cands[i].gi;
                basync = cands[i].async;
                bl = l2;
            }
            dr_status s = search_lines(P->fold2_R[cands[i].gi], run2(true), l2, ms[4], better);
            if (s != DR_OK) return s;
            if (better) {
                bgi = cands[i].gi;
                basync = cands[i].async;
                bl = l2;
            }
        }
        P->fold2_gi = bgi;
        P->fold2_async = basync;
        // triple-buffered strips on the best configuration (one barrier per
        // strip; three buffers, so a third fewer lines within the same memory)
        if (basync == 1) {
            P->fold2_async = 2;
            for (int c : {std::max(1, 2 * bl / 3), bl}) {
                double t = 1e30;
                dr_status s = run2(true)(c, t);
                if (s != DR_OK) return s;
                if (t < ms[4]) {
                    ms[4] = t;
                    basync = 2;
                    bl = c;
                }
            }
            P->fold2_async = basync;
        }
        // TMA-staged strips, two buffers on mbarriers (float coefficient
        // groups of whole 16-byte rows): the copies leave the threads'
        // instruction stream; two buffers share twice the strip budget
        // (every CTA shape: the copies free registers and issue slots, which
        // can move the best shape), at the tallest strips two buffers hold
        // and at half that
        if (P->m % 4 == 0) {
            const int keep_gi = P->fold2_gi, keep_async = P->fold2_async;
            bool won = false;
            for (int gi = 0; gi < kFold2Configs; ++gi) {
                if (!gi_ok(gi)) continue;
                P->fold2_gi = gi;
                P->fold2_async = 3;
                const int rt = std::max(1, P->fold2_Rt[gi]);
                for (int c : {rt, std::max(1, rt / 2)}) {
                    double t = 1e30;
                    dr_status s = run2(true)(c, t);
                    if (s != DR_OK) return s;
                    if (t < ms[4]) {
                        ms[4] = t;
                        bl = c;
                        bgi = gi;
                        won = true;
                    }
                    if (rt == 1) break;
                }
            }
            P->fold2_gi = won ? bgi : keep_gi;
            basync = won ? 3 : keep_async;
            P->fold2_async = basync;
        }
        // smaller angle blocks (more CTAs, each with less work): a fuller last wave
        {
            int bbv = 0;
            for (int v = 1; v < kFold2BlockVariants && P->d_fold2_blocks[bgi][v]; ++v) {
                P->fold2_bv = v;
                double t = 1e30;
                dr_status s = run2(true)(bl, t);
                if (s != DR_OK) return s;
                if (t < ms[4]) {
                    ms[4] = t;
                    bbv = v;
                }
            }
            P->fold2_bv = bbv;
        }
        // grids of a few waves leave SMs idle in the last one: try splitting the
        // march into line chunks (more CTAs; the distribution adds the partial sums)
        const long long ctas = (long long)P->fold2_nblocks[bgi][P->fold2_bv] * P->fold2_nchunk[bgi] * P->nz *
                               ((P->m + fold_static_mc(bgi) - 1) / fold_static_mc(bgi));
        if (!P->split_off && ctas < 4LL * P->num_sms * fold_static_min_blocks(bgi)) {
            const size_t chunk = sizeof(float) * (size_t)P->nz * P->fold_U * P->ns * ((P->m + 3) / 4 * 4);
            int bs = 1, bbv = P->fold2_bv;
            const int l0 = bl, bv0 = P->fold2_bv;
            for (int ns2 = 2; ns2 <= 4 && chunk * ns2 <= kSplitScratchMax; ++ns2) {
                P->fold2_split = ns2;
                // chunks change the wave count: block sizes are searched with them
                for (int v = 0; v < kFold2BlockVariants && P->d_fold2_blocks[bgi][v]; ++v) {
                    if (v != 0 && v != bv0 && v != 1) continue;
                    P->fold2_bv = v;
                    for (int c : {l0, std::max(1, l0 / 2)}) {
                        double t = 1e30;
                        dr_status s = run2(true)(c, t);
                        if (s != DR_OK) return s;
                        if (t < ms[4]) {
                            ms[4] = t;
                            bs = ns2;
                            bl = c;
                            bbv = v;
                        }
                        if (l0 == 1) break;
                    }
                }
            }
            P->fold2_split = bs;
            P->fold2_bv = bbv;
            // keep exactly the chosen chunks' scratch (the trials grew it to the largest)
            const size_t keep = bs > 1 ? chunk * bs : 0;
            if (P->d_ru_split && P->ru_split_bytes != keep) {
                cudaFree(P->d_ru_split);
                P->d_ru_split = nullptr;
                P->ru_split_bytes = 0;
                if (keep) {
                    dr_status s = ensure_split_scratch(P, keep);
                    if (s != DR_OK) return s;
                }
            }
        }
        // confirm the strip height against its neighbours with more timed
        // launches (neighbouring heights often differ by less than the noise
        // of the short trials above)
        {
            const int all[] = {1, 2, 3, 4, 6, 8, 12, 16};
            int bi = 0;
            while (bi < 7 && all[bi] != bl) ++bi;
            double best_t = 1e30;
            int best_c = bl;
            for (int i : {bi - 1, bi, bi + 1}) {
                const int cap = P->fold2_async == 3 ? P->fold2_Rt[bgi] : P->fold2_R[bgi];
                if (i < 0 || i > 7 || all[i] > cap) continue;
                double t = 1e30;
                dr_status s = run2(true, 6)(all[i], t);
                if (s != DR_OK) return s;
                if (t < best_t) {
                    best_t = t;
                    best_c = all[i];
                }
            }
            if (best_t < 1e30) {
                bl = best_c;
                ms[4] = best_t;  // the chosen configuration's confirmed time
            }
        }
        P->fold2_lines = bl;
        P->fold2_lines_st = bl;
        P->fold2_async_st = P->fold2_async;
        P->fold2_gi_st = bgi;
        if (P->prec == DR_BF16_F32ACC) {
            // storage-typed calls march bf16 strips: the compute-typed group and
            // its 8-coefficient partner (same CTA shape), whose 16-byte bf16
            // pixel vectors load like the 4-coefficient float ones
            double best_t = 1e30;
            int bls = bl, bas = 0, bgs = bgi;
            int cand[2] = {bgi, -1};
            if ((bgi | 1) != bgi && gi_ok(bgi | 1)) cand[1] = bgi | 1;
            for (int gs : cand) {
                if (gs < 0) continue;
                P->fold2_gi_st = gs;
                for (int as = 0; as < (gs == bgi ? 3 : 2); ++as) {
                    P->fold2_async_st = as;
                    int lines = bls;
                    dr_status s = search_lines(P->fold2_R[gs], run2(false), lines, best_t, better);
                    if (s != DR_OK) return s;
                    if (better) {
                        bas = as;
                        bls = lines;
                        bgs = gs;
                    }
                }
            }
            P->fold2_gi_st = bgs;
            P->fold2_lines_st = bls;
            P->fold2_async_st = bas;
            ms_st2 = best_t;
        }
    }
    if (P->prec == DR_BF16_F32ACC) {
        // storage-typed calls of BF16 plans run the bf16-strip kernels: their own choice
        double ms_st0 = 1e30;
        dr_status s0 = time_fwd(0, ms_st0, false, 2);
        if (s0 != DR_OK) return s0;
        int best = 0;
        double bt = ms_st0;
        if (ms_st1 < bt) { best = 1; bt = ms_st1; }
        if (ms_st2 < bt) { best = 2; bt = ms_st2; }
        P->sel_fwd_st = best;
    }
    auto time_adj = [&](int v, double &best, int reps = 3) -> dr_status {
        if (canceled()) return fail(DR_ECANCELED, "autotune: canceled");
        for (int rep = 0; rep < reps; ++rep) {
            DR_CUDA_TRY(cudaEventRecord(e0, st));
            dr_status s = launch_adj_variant(P, v, true, g_scratch, u_scratch, 1.0, 0.0, true, st);
            if (s != DR_OK) return s;
            DR_CUDA_TRY(cudaEventRecord(e1, st));
            DR_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.f;
            DR_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            if (rep > 0) best = std::min(best, (double)t);
        }
        return DR_OK;
    };
    {
        dr_status s = time_adj(0, ms[2], 2);
        if (s != DR_OK) return s;
    }
    if (P->fold_U > 0) {
        // folded adjoint: distinct angles per pipeline stage (8, 7, 6: smaller
        // windows let more CTAs share an SM; the summation order is the same)
        int best_pp = 8;
        for (int pp : {8, 7, 6}) {
            P->fold_adj_pp = pp;
            double t = 1e30;
            dr_status s = time_adj(1, t);
            if (s != DR_OK) return s;
            if (t < ms[3]) {
                ms[3] = t;
                best_pp = pp;
            }
        }
        P->fold_adj_pp = best_pp;
    }
    for (int i = 0; i < 5; ++i) P->tune_ms[i] = ms[i] < 1e29 ? ms[i] : -1.0;
    {
        int best = 0;
        if (ms[1] < ms[best]) best = 1;
        if (ms[4] < (best == 1 ? ms[1] : ms[0])) best = 2;
        P->sel_fwd = best;
        if (P->prec != DR_BF16_F32ACC) P->sel_fwd_st = best;
    }
    P->sel_adj = ms[3] < ms[2] ? 1 : 0;
    P->tuned = true;
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto ins = g_tune_cache.emplace(key, TuneVal{P->sel_fwd, P->sel_adj, P->fold_lines, P->fold_async,
                                                 P->fold_lines_st, P->fold_async_st, P->fold2_gi, P->fold2_lines,
                                                 P->fold2_lines_st, P->sel_fwd_st, P->fold2_split,
                                                 P->fold2_async, P->fold2_async_st, P->fold_adj_pp, P->fold2_bv,
                                                 P->fold2_gi_st, {0, 0, 0, 0, 0}});
    if (ins.second) {
        for (int i = 0; i < 5; ++i) ins.first->second.ms[i] = P->tune_ms[i];
    } else {  // another thread tuned the same problem first: follow its choice
        P->sel_fwd = ins.first->second.fwd;
        P->sel_adj = ins.first->second.adj;
        P->fold_lines = ins.first->second.lines;
        P->fold_async = ins.first->second.async;
        P->fold_lines_st = ins.first->second.lines_st;
        P->fold_async_st = ins.first->second.async_st;
        P->fold2_gi = ins.first->second.f2_gi;
        P->fold2_gi_st = ins.first->second.f2_gi_st;
        P->fold2_lines = ins.first->second.f2_lines;
        P->fold2_lines_st = ins.first->second.f2_lines_st;
        P->sel_fwd_st = ins.first->second.fwd_st;
        P->fold2_split = P->split_off ? 1 : ins.first->second.f2_split;
        P->fold2_async = ins.first->second.f2_async;
        P->fold2_async_st = ins.first->second.f2_async_st;
        P->fold_adj_pp = ins.first->second.adj_pp;
        P->fold2_bv = ins.first->second.f2_bv;
    }
    return DR_OK;
}

}  // namespace dr

using namespace dr;

extern "C" {

dr_status dyn_radon_fwd(dr_plan *P, const void *u, void *g) {
    clear_error();
    if (!P || !u || !g) return fail(DR_EINVAL, "dyn_radon_fwd: NULL argument");
    return launch_fwd(P, u, g, nullptr, 0, 0.0, P->stream);
}

dr_status dyn_radon_adj(dr_plan *P, const void *g, void *u, double beta) {
    clear_error();
    if (!P || !u || !g) return fail(DR_EINVAL, "dyn_radon_adj: NULL argument");
    if (!std::isfinite(beta)) return fail(DR_EINVAL, "dyn_radon_adj: beta must be finite");
    return launch_adj(P, g, u, 1.0, beta, false, P->stream);
}

dr_status dr_plan_set_variant(dr_plan *P, int fwd_variant, int adj_variant) {
    clear_error();
    if (!P) return fail(DR_EINVAL, "dr_plan_set_variant: NULL plan");
    if (fwd_variant < -1 || fwd_variant > 2 || adj_variant < -1 || adj_variant > 1)
        return fail(DR_EINVAL, "dr_plan_set_variant: forward variants are -1 (auto), 0 (direct), 1 (fold) or 2 "
                               "(fold in two kernels); adjoint variants -1, 0 or 1");
    if ((fwd_variant == 1 && !(P->fold_U > 0 && P->fold_fwd_ok)) || (adj_variant == 1 && P->fold_U == 0) ||
        (fwd_variant == 2 && !(P->fold_U > 0 && P->fold2_ok)))
        return fail(DR_EINVAL, "dr_plan_set_variant: the half-turn fold is unavailable for this plan");
    P->var_fwd = fwd_variant;
    P->var_adj = adj_variant;
    return DR_OK;
}

dr_status dr_plan_autotune(dr_plan *P, double *times_ms) {
    clear_error();
    if (!P) return fail(DR_EINVAL, "dr_plan_autotune: NULL plan");
    if (!P->tuned) {
        const size_t cs = calc_size(P->prec);
        void *us = nullptr, *gs = nullptr;
        DR_CUDA_TRY(cudaMalloc(&us, std::max<size_t>(nu_elems(P) * cs, 16)));
        cudaError_t e = cudaMalloc(&gs, std::max<size_t>(ng_elems(P) * cs, 16));
        if (e != cudaSuccess) {
            cudaFree(us);
            return cuda_fail(e, "dr_plan_autotune: scratch");
        }
        dr_status s = autotune(P, us, gs);
        cudaStreamSynchronize(P->graph_stream);
        cudaFree(us);
        cudaFree(gs);
        if (s != DR_OK) return s;
    }
    if (times_ms)
        for (int i = 0; i < 5; ++i) times_ms[i] = P->tune_ms[i];
    return DR_OK;
}

dr_status dr_plan_set_fold_strip(dr_plan *P, int lines, int async) {
    clear_error();
    if (!P) return fail(DR_EINVAL, "dr_plan_set_fold_strip: NULL plan");
    if (!(P->fold_U > 0 && P->fold_fwd_ok)) return fail(DR_EINVAL, "dr_plan_set_fold_strip: no folded forward");
    const int async_ok = P->m == P->M && ((P->prec == DR_F32 && P->M % 4 == 0) ||
                                          (P->prec == DR_BF16_F32ACC && P->M % 8 == 0));
    if (lines < 1 || (async != 0 && async != 1) || (async && !async_ok) || (async ? 2 : 1) * lines > P->fold_R)
        return fail(DR_EINVAL, "dr_plan_set_fold_strip: lines must be in [1, " + std::to_string(P->fold_R) +
                                   "] (half that with async), async only for whole 16-byte vectors");
    P->fold_lines = P->fold_lines_st = lines;
    P->fold_async = P->fold_async_st = async;
    return DR_OK;
}

dr_status dr_plan_set_fold_groups(dr_plan *P, int group, int threads, int rays_per_thread, int lines) {
    clear_error();
    if (!P) return fail(DR_EINVAL, "dr_plan_set_fold_groups: NULL plan");
    if (!(P->fold_U > 0 && P->fold2_ok)) return fail(DR_EINVAL, "dr_plan_set_fold_groups: variant unavailable");
    // the configuration with this group and CTA size, and these rays per thread
    // (0: the most rays per thread that configuration family has)
    int gi = -1;
    for (int c = 0; c < kFold2Configs; ++c)
        if (fold_static_mc(c) == group && fold_static_threads(c) == threads &&
            (rays_per_thread == 0 ? (gi < 0 || fold_static_rpt_gi(c) > fold_static_rpt_gi(gi))
                                  : fold_static_rpt_gi(c) == rays_per_thread))
            gi = c;
    if (gi < 0 || (group == 8 && P->m <= 4) || lines < 1 || lines > std::max(P->fold2_R[gi], P->fold2_Rt[gi]) ||
        (size_t)P->nz * ((P->m + group - 1) / group) > 65535)
        return fail(DR_EINVAL, "dr_plan_set_fold_groups: no such configuration (group 4 or 8, 8 only for m > 4; "
                               "threads 256, 512 or 1024 with their rays per thread) or lines outside the strip "
                               "budget");
    P->fold2_gi = P->fold2_gi_st = gi;
    P->fold2_lines = P->fold2_lines_st = lines;
    P->fold2_bv = 0;
    return DR_OK;
}

dr_status dr_plan_set_fold_march(dr_plan *P, int nsplit, int async) {
    clear_error();
    if (!P) return fail(DR_EINVAL, "dr_plan_set_fold_march: NULL plan");
    if (!(P->fold_U > 0 && P->fold2_ok)) return fail(DR_EINVAL, "dr_plan_set_fold_march: variant unavailable");
    if (nsplit < 1 || nsplit > 8 || async < 0 || async > 3)
        return fail(DR_EINVAL, "dr_plan_set_fold_march: nsplit must be 1..8 and async 0, 1, 2 or 3");
    P->fold2_split = nsplit;
    P->fold2_async = P->fold2_async_st = async;
    return DR_OK;
}

dr_status dr_plan_set_fold_blocks(dr_plan *P, int extra) {
    clear_error();
    if (!P) return fail(DR_EINVAL, "dr_plan_set_fold_blocks: NULL plan");
    if (!(P->fold_U > 0 && P->fold2_ok)) return fail(DR_EINVAL, "dr_plan_set_fold_blocks: variant unavailable");
    if (extra < 0 || extra >= kFold2BlockVariants || !P->d_fold2_blocks[P->fold2_gi][extra])
        return fail(DR_EINVAL, "dr_plan_set_fold_blocks: no such block variant for this plan and group");
    P->fold2_bv = extra;
    return DR_OK;
}

dr_status dr_plan_set_fold_adj_stage(dr_plan *P, int angles) {
    clear_error();
    if (!P) return fail(DR_EINVAL, "dr_plan_set_fold_adj_stage: NULL plan");
    if (P->fold_U == 0) return fail(DR_EINVAL, "dr_plan_set_fold_adj_stage: no folded adjoint");
    if (angles < 1 || angles > 32) return fail(DR_EINVAL, "dr_plan_set_fold_adj_stage: angles must be 1..32");
    P->fold_adj_pp = angles;
    return DR_OK;
}

dr_status dr_plan_info(const dr_plan *P, dr_plan_info_t *info) {
    clear_error();
    if (!P || !info) return fail(DR_EINVAL, "dr_plan_info: NULL argument");
    info->unique_angles = P->fold_U;
    info->max_group = P->fold_maxgrp;
    info->fwd_variant = P->var_fwd >= 0 ? P->var_fwd : P->sel_fwd;
    info->adj_variant = P->var_adj >= 0 ? P->var_adj : P->sel_adj;
    info->tuned = P->tuned ? 1 : 0;
    info->device_bytes = P->table_bytes + P->ws.bytes + (P->d_gt ? P->gt_bytes : 0) + P->fbp_bytes +
                         P->ru_split_bytes;
    info->fold_lines = P->fold_lines;
    info->fold_async = P->fold_async;
    info->fold2_group = P->fold2_ok ? fold_static_mc(P->fold2_gi) : 0;
    info->fold2_threads = P->fold2_ok ? fold_static_threads(P->fold2_gi) : 0;
    info->fold2_rays_per_thread = P->fold2_ok ? fold_static_rpt_gi(P->fold2_gi) : 0;
    info->fold2_lines = P->fold2_ok ? P->fold2_lines : 0;
    info->fold2_split = P->fold2_ok ? P->fold2_split : 0;
    info->fold2_async = P->fold2_ok ? P->fold2_async : 0;
    info->fold_adj_angles = P->fold_U > 0 ? P->fold_adj_pp : 0;
    info->fold2_angles =
        P->fold2_ok ? P->fold2_P[P->fold2_gi][P->d_fold2_blocks[P->fold2_gi][P->fold2_bv] ? P->fold2_bv : 0] : 0;
    info->fwd_variant_storage = P->var_fwd >= 0 ? P->var_fwd : P->sel_fwd_st;
    return DR_OK;
}

}  // extern "C"
