// ragged.cu -- spec_ragged: many traces that each bring their own length,
// band, point count, decimation and taps, transformed in one call.
//
// The first call with a given descriptor list builds a plan and caches it in
// the context:
//   * every descriptor is validated exactly as the single-shape entry point
//     would validate it (Section 2.1-2.3 conventions, include/spec.h);
//   * each transform kind runs as one persistent launch over a work queue: a
//     device array of units (a few traces of one shape, or a part of one long
//     trace), sorted largest first and popped from an atomic counter by one
//     CTA per SM (FFT: k_fft_queue; chirp-z: k_czt_queue, with the chirps
//     evaluated in the kernel and one FFT(v)/L table per distinct (N, M,
//     band); Zoom: k_zoom_queue);
//   * traces outside a queue's sizes (FFT residue FFTs above 4096 points,
//     Zoom K above 16384) are grouped into classes of one kernel shape and
//     launched as before, on parallel branches of the same graph;
//   * the autotuner times the alternatives a plan admits (FFT queue: long
//     traces through a per-CTA workspace or as residue-pair units; FFT
//     classes: lanes, pass radix, cluster kernel) and keeps the fastest;
//   * one CUDA graph is captured (counter reset, queue launch, class
//     branches), so the whole batch is one graph launch.
// Later calls with the same descriptors replay the graph (re-captured if the
// pool pointers change).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <tuple>
#include <vector>

#include "ctx.h"
#include "fft_block.cuh"
#include "spec.h"
#include "spec_internal.h"

using namespace spec;

struct RaggedClass {
    int path = 0;        // 0 FFT, 1 CZT, 2 Zoom (one CTA), 3 Zoom pruned cluster FFT (after the FIR)
    int K = 0, L = 0;
    FftPlan fp;          // FFT (path 0) or pruned complex FFT (path 3)
    int lanes = 1;
    bool in_queue = false;   // the work queue covers these traces too
    size_t smem = 0;     // Zoom one-CTA: the largest need in the class
    bool lo4 = false;    // Zoom one-CTA: every trace has L_out <= K/4 (sparse first FFT pass)
    int64_t first = 0, count = 0;
    const float2* tab = nullptr;
    float tuned_us = 0.f;
};

struct RaggedPlan {
    int kind = 0;
    double fs = 0.0;
    std::vector<spec_desc> descs;
    std::vector<RaggedClass> classes;
    RaggedItem* items = nullptr;
    int64_t fir_first = 0, fir_count = 0;
    int fir_chunks = 0;
    size_t fir_smem = 0;
    float2* tables = nullptr;
    float2* work = nullptr;
    // work queue (chirp-z: CztUnit; FFT: FftUnit), its length, the counter;
    // chirp-z: `tables` holds the FFT(v)/L pool
    void* units = nullptr;
    int nunits = 0;
    size_t qsmem = 0;          // Zoom queue: dynamic shared memory of the launch
    bool use_queue = false;    // the captured graph runs the queue (else the per-shape classes)
    float t_queue_us = 0.f, t_classes_us = 0.f;   // the two forms as timed when the plan was built
    float2* vpool = nullptr;   // chirp-z queue: FFT(v)/L per distinct (N, M, band)
    float2* qws = nullptr;     // FFT queue: per-CTA workspaces (mode 2 units)
    int64_t qws_per = 0;
    void* units_alt = nullptr; // FFT queue: the same work as residue-pair units (timed against `units`)
    int nunits_alt = 0;
    unsigned* counter = nullptr;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;
    cudaGraphExec_t exec = nullptr;
    const void* gx = nullptr;
    const void* gt = nullptr;
    void* gX = nullptr;
};

void ragged_plan_free(RaggedPlan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    for (auto s : p->side) cudaStreamDestroy(s);
    for (auto e : p->ev) cudaEventDestroy(e);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->items) cudaFree(p->items);
    if (p->tables) cudaFree(p->tables);
    if (p->work) cudaFree(p->work);
    if (p->units) cudaFree(p->units);
    if (p->units_alt) cudaFree(p->units_alt);
    if (p->qws) cudaFree(p->qws);
    if (p->vpool) cudaFree(p->vpool);
    if (p->counter) cudaFree(p->counter);
    delete p;
}

namespace {

bool same_descs(const RaggedPlan* p, int kind, double fs, const spec_desc* d, int64_t count) {
    return p->kind == kind && p->fs == fs && (int64_t)p->descs.size() == count &&
           (count == 0 || std::memcmp(p->descs.data(), d, (size_t)count * sizeof(spec_desc)) == 0);
}

const float2* tw_for(spec_ctx* c, int LF, int emax = 16) { return c->block_tw + block_twiddle_offset(LF, emax); }

constexpr int kQueueThreads = 256;    // threads of the persistent FFT kernel's CTA (two per SM)

cudaError_t launch_class(spec_ctx* c, RaggedPlan* P, const RaggedClass& k, cudaStream_t s, const float* x,
                         const float* taps, float2* X) {
    const RaggedItem* it = P->items + k.first;
    switch (k.path) {
        case 0:
            return fft_launch(k.fp, x, k.count, 0, 0, tw_for(c, k.fp.LZ, k.fp.emax), k.tab, X, 0, s, k.lanes, it);
        case 1:
            return czt_ragged_launch(k.L, it, k.count, x, P->tables, tw_for(c, k.L), X, s);
        case 2:
            return zoom_ragged_launch(k.K, it, k.count, k.smem, x, taps, tw_for(c, k.K), X, s, k.lo4);
        default:
            return c2c_launch(k.fp, P->work, 0, 0, k.count, k.K / 2, tw_for(c, k.fp.LZ), k.tab, X, 0, s, it);
    }
}

// Time one class (median of 3 after a warm-up) on the capture stream.
float time_class(spec_ctx* c, RaggedPlan* P, const RaggedClass& k, const float* x, const float* taps, float2* X) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {
        cudaEventRecord(a, P->cap);
        if (launch_class(c, P, k, P->cap, x, taps, X) != cudaSuccess) {
            best = 1e30f;
            break;
        }
        cudaEventRecord(b, P->cap);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (r > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaGetLastError();
    return best;
}

spec_status capture(spec_ctx* c, RaggedPlan* P, const float* x, const float* taps, float2* X) {
    if (P->exec) {
        cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
    }
    const size_t nbr = P->classes.size() + 1;
    while (P->side.size() < nbr) {
        cudaStream_t s;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) return ctx_cuda_fail(c, e, "ragged streams");
        P->side.push_back(s);
    }
    while (P->ev.size() < nbr + 1) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return ctx_cuda_fail(c, e, "ragged events");
        P->ev.push_back(ev);
    }
    cudaError_t e = cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return ctx_cuda_fail(c, e, "graph capture");
    cudaError_t le = cudaEventRecord(P->ev[0], P->cap);
    if (P->use_queue && P->nunits > 0 && le == cudaSuccess) {
        // one persistent launch over the unit queue
        le = cudaMemsetAsync(P->counter, 0, sizeof(unsigned), P->cap);
        if (le == cudaSuccess && P->kind == SPEC_KIND_CZT)
            le = czt_queue_launch(P->items, (const CztUnit*)P->units, P->nunits, P->counter, x, P->vpool,
                                  c->block_tw, c->block_tw + block_twiddle_offset(64, 32) - fft_twiddle_offset(64, 32),
                                  X, c->sms, P->cap);
        if (le == cudaSuccess && P->kind == SPEC_KIND_ZOOM)
            le = zoom_queue_launch(P->items, (const ZoomUnit*)P->units, P->nunits, P->counter, P->qsmem, x, taps,
                                   c->block_tw, X, c->sms, P->cap);
        if (le == cudaSuccess && P->kind == SPEC_KIND_FFT)
            le = fft_queue_launch(P->items, (const FftUnit*)P->units, P->nunits, P->counter, x, c->block_tw, X,
                                  P->qws, P->qws_per, 2 * std::max(1, c->sms), P->cap);
    }
    size_t br = 0;
    // one branch per class of paths 0-2; the large Zoom path (FIR, then its
    // pruned-FFT classes) forms one more branch
    for (const RaggedClass& k : P->classes) {
        if (k.path == 3 || le != cudaSuccess || (P->use_queue && k.in_queue)) continue;
        cudaStream_t s = P->side[br];
        le = cudaStreamWaitEvent(s, P->ev[0], 0);
        if (le == cudaSuccess) le = launch_class(c, P, k, s, x, taps, X);
        if (le == cudaSuccess) le = cudaEventRecord(P->ev[br + 1], s);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(P->cap, P->ev[br + 1], 0);
        ++br;
    }
    if (P->fir_count > 0 && le == cudaSuccess) {
        cudaStream_t s = P->side[br];
        le = cudaStreamWaitEvent(s, P->ev[0], 0);
        if (le == cudaSuccess)
            le = zoom_fir_ragged_launch(P->items + P->fir_first, P->fir_count, P->fir_chunks, P->fir_smem, x, taps,
                                        P->work, s);
        for (const RaggedClass& k : P->classes)
            if (k.path == 3 && le == cudaSuccess) le = launch_class(c, P, k, s, x, taps, X);
        if (le == cudaSuccess) le = cudaEventRecord(P->ev[br + 1], s);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(P->cap, P->ev[br + 1], 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(P->cap, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return ctx_cuda_fail(c, le != cudaSuccess ? le : e, "graph capture");
    }
    e = cudaGraphInstantiate(&P->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return ctx_cuda_fail(c, e, "graph instantiate");
    P->gx = x;
    P->gt = taps;
    P->gX = X;
    return SPEC_OK;
}

spec_status build_plan(spec_ctx* c, int kind, const spec_desc* d, int64_t count, double fs, const float* x,
                       const float* taps, float2* X, RaggedPlan** out) {
    RaggedPlan* P = new RaggedPlan();
    P->kind = kind;
    P->fs = fs;
    P->descs.assign(d, d + count);
    auto bail = [&](spec_status s) {
        ragged_plan_free(P);
        return s;
    };
    // ---- validate and classify ---------------------------------------------
    struct Tmp {
        int64_t idx;
        RaggedItem it;
    };
    std::map<std::tuple<int, int, int>, std::vector<Tmp>> groups;   // (path, key1, key2)
    std::map<std::tuple<int, int, int>, FftPlan> gplan;
    std::map<std::tuple<int, int, int>, size_t> gsmem;
    for (int64_t i = 0; i < count; ++i) {
        const spec_desc& q = d[i];
        std::string why;
        const std::string at = "descriptor " + std::to_string(i) + ": ";
        if (q.n < 1 || q.n > (int64_t(1) << 24) || q.x_off < 0 || q.out_off < 0)
            return bail(ctx_fail(c, SPEC_EINVAL, at + "n must be in [1, 2^24] and offsets >= 0"));
        RaggedItem it = {};
        it.x_off = q.x_off;
        it.out_off = q.out_off;
        it.n = (int32_t)q.n;
        if (kind == SPEC_KIND_FFT) {
            if (q.n_fft < q.n || q.n_fft > (int64_t(1) << 24) || !is_pow2(q.n_fft))
                return bail(ctx_fail(c, SPEC_EINVAL, at + "n_fft must be a power of two >= n"));
            FftPlan p;
            if (q.n_fft < 32 || !fft_plan(1, q.n, q.n_fft, &p, &why))
                return bail(ctx_fail(c, SPEC_EUNSUPPORTED, at + (why.empty() ? "n_fft below 32" : why)));
            groups[{0, p.H, p.LZ}].push_back({i, it});
        } else if (kind == SPEC_KIND_CZT) {
            if (q.m < 1 || q.m > (int64_t(1) << 24) || !std::isfinite(q.f1) || !std::isfinite(q.f2))
                return bail(ctx_fail(c, SPEC_EINVAL, at + "m must be >= 1 and f1, f2 finite"));
            if (!czt_supported(q.n, q.m, &why)) return bail(ctx_fail(c, SPEC_EUNSUPPORTED, at + why));
            const double step = q.m > 1 ? (q.f2 - q.f1) / (double)(q.m - 1) : 0.0;
            it.A = cycles_to_fixed(q.f1 / fs);
            it.B = cycles_to_fixed(0.5 * (step / fs));
            it.m = (int32_t)q.m;
            groups[{1, czt_length(q.n, q.m), 0}].push_back({i, it});
        } else {
            if (q.d < 1 || q.n_fft < 1 || q.n_fft % q.d != 0 || !is_pow2(q.n_fft / q.d) || q.n_taps < 1 ||
                q.n_taps > 65536 || q.taps_off < 0 || !std::isfinite(q.f1) || !std::isfinite(q.f2))
                return bail(ctx_fail(c, SPEC_EINVAL, at + "invalid d, n_fft, taps or band"));
            const int64_t K = q.n_fft / q.d;
            const int64_t lout = (q.n + q.n_taps - 1 + q.d - 1) / q.d;
            if (lout > K) return bail(ctx_fail(c, SPEC_EINVAL, at + "ceil((n + n_taps - 1)/d) exceeds n_fft/d"));
            it.d = (int32_t)q.d;
            it.n_taps = (int32_t)q.n_taps;
            it.lout = (int32_t)lout;
            it.tab_off = q.taps_off;
            it.A = cycles_to_fixed(0.5 * (q.f1 + q.f2) / fs);
            ZoomPlan zp;
            std::string w1, w2;
            if (zoom_plan(q.n, q.d, q.n_taps, q.n_fft, fs, q.f1, q.f2, &zp, &w1)) {
                it.rs = zoom_rows(lout, q.n_taps, q.d);
                auto key = std::make_tuple(2, (int)K, 0);
                groups[key].push_back({i, it});
                gsmem[key] = std::max(gsmem[key], zoom_smem_for(it.n_taps, it.d, it.rs, (int)K));
            } else if (zoom_big_plan(1, q.n, q.d, q.n_taps, q.n_fft, fs, q.f1, q.f2, &zp, &w2)) {
                it.rs = fir_rows(q.n_taps, q.d);
                groups[{3, (int)K, zp.fft.LZ}].push_back({i, it});
                P->fir_smem = std::max(P->fir_smem, fir_smem_for(it.n_taps, it.d));
                P->fir_chunks = std::max<int>(P->fir_chunks, (int)((lout + fir_chunk() - 1) / fir_chunk()));
            } else {
                return bail(ctx_fail(c, SPEC_EUNSUPPORTED, at + w1 + "; " + w2));
            }
        }
    }
    // ---- items, per class, large-zoom classes last ---------------------------
    std::vector<RaggedItem> items;
    items.reserve((size_t)count);
    int64_t tab_total = 0, work_total = 0, vp_total = 0;
    // shapes the work queue covers; their classes are built too, and the plan
    // keeps whichever of the two graphs (queue or per-shape launches) is faster
    std::set<std::tuple<int, int, int>> queued;
    std::vector<CztUnit> units;
    std::map<int, std::vector<RaggedItem>> vkeys;      // per L: one item per distinct (N, M, B)
    std::vector<FftUnit> funits, funits_pairs;
    int64_t ws_per = 0;
    std::vector<ZoomUnit> zunits;
    size_t zsmem = 0;
    if (kind == SPEC_KIND_ZOOM) {
        // work queue for the one-CTA Zoom classes K in [64, 16384]: units of
        // traces of one K, as many as their shared-memory slices allow
        const size_t budget = 227 * 1024 - 1024;
        for (auto g = groups.rbegin(); g != groups.rend();) {
            const int path = std::get<0>(g->first), K = std::get<1>(g->first);
            if (path != 2 || K < 64 || K > 16384) {
                ++g;
                continue;
            }
            std::vector<Tmp>& tr = g->second;
            auto need = [&](const Tmp& x) {
                return (zoom_smem_for(x.it.n_taps, x.it.d, x.it.rs, K) + 15) & ~(size_t)15;
            };
            std::stable_sort(tr.begin(), tr.end(), [&](const Tmp& p1, const Tmp& p2) { return need(p1) > need(p2); });
            const int G = zoom_queue_groups(K);
            const size_t scratch = ((size_t)padded_len(K) * sizeof(float2) + 15) & ~(size_t)15;
            size_t j = 0;
            while (j < tr.size()) {
                const size_t slice = need(tr[j]);                  // largest need of the unit (sorted)
                int F = (int)std::min<size_t>((size_t)G, budget / slice);
                if (F < G || tr.size() - j < (size_t)G) {
                    // some groups idle: keep room for the scratch FFT area
                    F = (int)std::min<size_t>((size_t)F, (budget - scratch) / slice);
                }
                if (F < 1) return bail(ctx_fail(c, SPEC_EUNSUPPORTED, "zoom: a trace exceeds the queue's shared memory"));
                const int cnt = (int)std::min<size_t>((size_t)F, tr.size() - j);
                ZoomUnit zu{K, (int)items.size(), cnt, F, (int)slice, (int)(F * slice)};
                zsmem = std::max(zsmem, cnt < G ? F * slice + scratch : F * slice);
                zunits.push_back(zu);
                for (int q = 0; q < cnt; ++q) items.push_back(tr[j + q].it);
                j += cnt;
            }
            queued.insert(g->first);
            ++g;
        }
    }
    if (kind == SPEC_KIND_FFT) {
        // work queue for every (H, LZ) the persistent kernel handles: whole
        // traces per unit up to H = 16384, residue pairs of one trace above;
        // largest LZ (then H) first, a trace's units adjacent
        for (auto g = groups.rbegin(); g != groups.rend();) {
            const int H = std::get<1>(g->first), LZ = std::get<2>(g->first);
            const int R = H / LZ;
            FftPlan fp;
            std::string why;
            const bool ok = LZ >= 16 && LZ <= 4096 && R >= 2 && H >= 32 &&
                            fft_plan(1, 2 * (int64_t)LZ, 2 * (int64_t)H, &fp, &why) && fp.emax == 16 && fp.E == 16;
            if (!ok) {
                ++g;
                continue;
            }
            const float2* tab = nullptr;
            spec_status ts = ctx_plan_table(c, 0, fp, &tab);
            if (ts != SPEC_OK) return bail(ts);
            const int T = LZ / 16;
            if ((R / 2) * T <= kQueueThreads) {
                const int F = kQueueThreads / ((R / 2) * T);
                for (size_t j = 0; j < g->second.size(); ++j) {
                    if (j % F == 0) {
                        funits.push_back(FftUnit{tab, LZ, ilog2(R), (int)items.size(), 0, 0, 0});
                        funits_pairs.push_back(funits.back());
                    }
                    ++funits.back().count;
                    ++funits_pairs.back().count;
                    items.push_back(g->second[j].it);
                }
            } else {
                // one trace per unit through the CTA's workspace (mode 2); the
                // alternative list splits it into residue-pair units (mode 1)
                const int G = kQueueThreads / T;
                for (Tmp& tr : g->second) {
                    funits.push_back(FftUnit{tab, LZ, ilog2(R), (int)items.size(), 1, 0, 2});
                    for (int g0 = 0; g0 < R / 2; g0 += G)
                        funits_pairs.push_back(
                            FftUnit{tab, LZ, ilog2(R), (int)items.size(), std::min(G, R / 2 - g0), g0, 1});
                    items.push_back(tr.it);
                }
                ws_per = std::max<int64_t>(ws_per, H);
            }
            queued.insert(g->first);
            ++g;
        }
    }
    if (kind == SPEC_KIND_CZT) {
        // work queue: units of 16384/L traces, largest L first; FFT(v)/L
        // shared by every trace with the same (N, M, B)
        std::map<std::tuple<int, int, uint64_t>, int64_t> voff;
        for (auto g = groups.rbegin(); g != groups.rend(); ++g) {
            const int L = std::get<1>(g->first);
            const int per = czt_queue_unit_traces(L);
            for (size_t j = 0; j < g->second.size(); ++j) {
                RaggedItem it = g->second[j].it;
                const auto key = std::make_tuple(it.n, it.m, it.B);
                auto f = voff.find(key);
                if (f == voff.end()) {
                    f = voff.emplace(key, vp_total).first;
                    RaggedItem kk = it;
                    kk.tab_off = vp_total;
                    vkeys[L].push_back(kk);
                    vp_total += L;
                }
                it.tab_off = f->second;
                if (j % per == 0) units.push_back(CztUnit{L, (int)items.size(), 0, 0});
                ++units.back().count;
                items.push_back(it);
            }
        }
        for (auto& kv : groups) queued.insert(kv.first);
    }
    for (auto& kv : groups) {
        const int path = std::get<0>(kv.first);
        RaggedClass k;
        k.path = path;
        k.first = (int64_t)items.size();
        k.count = (int64_t)kv.second.size();
        if (path == 0) {
            const spec_desc& q0 = d[kv.second[0].idx];
            std::string why;
            fft_plan(k.count, q0.n, q0.n_fft, &k.fp, &why);
        } else if (path == 1) {
            k.L = std::get<1>(kv.first);
        } else if (path == 2) {
            k.K = std::get<1>(kv.first);
            k.smem = gsmem[kv.first];
            k.lo4 = true;
            for (const Tmp& t : kv.second) k.lo4 = k.lo4 && (int64_t)t.it.lout * 4 <= k.K;
        } else {
            k.K = std::get<1>(kv.first);
            std::string why;
            c2c_plan(k.count, std::get<2>(kv.first), k.K, &k.fp, &why);
            // c2c_plan picked LZ from the largest possible input of the class
            k.fp.LZ = std::get<2>(kv.first);
            c2c_plan(k.count, k.fp.LZ, k.K, &k.fp, &why);
        }
        for (Tmp& t : kv.second) {
            if (path == 1) {
                t.it.tab_off = tab_total;
                tab_total += (int64_t)t.it.n + k.L + t.it.m;
            }
            if (path == 3) {
                t.it.u_off = work_total;
                work_total += k.fp.LZ;
            }
            items.push_back(t.it);
        }
        k.in_queue = queued.count(kv.first) > 0;
        P->classes.push_back(k);
    }
    for (const RaggedClass& k : P->classes)
        if (k.path == 3) {
            if (P->fir_count == 0) P->fir_first = k.first;
            P->fir_count += k.count;
        }
    cudaError_t e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess && !items.empty()) e = cudaMalloc(&P->items, items.size() * sizeof(RaggedItem));
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpy(P->items, items.data(), items.size() * sizeof(RaggedItem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && tab_total > 0) e = cudaMalloc(&P->tables, (size_t)tab_total * sizeof(float2));
    if (e == cudaSuccess && vp_total > 0) e = cudaMalloc(&P->vpool, (size_t)vp_total * sizeof(float2));
    if (e == cudaSuccess && work_total > 0) e = cudaMalloc(&P->work, (size_t)work_total * sizeof(float2));
    if (e == cudaSuccess && !zunits.empty()) {
        P->nunits = (int)zunits.size();
        P->qsmem = zsmem;
        e = cudaMalloc(&P->units, zunits.size() * sizeof(ZoomUnit));
        if (e == cudaSuccess)
            e = cudaMemcpy(P->units, zunits.data(), zunits.size() * sizeof(ZoomUnit), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&P->counter, sizeof(unsigned));
    }
    if (e == cudaSuccess && !funits.empty()) {
        P->nunits = (int)funits.size();
        e = cudaMalloc(&P->units, funits.size() * sizeof(FftUnit));
        if (e == cudaSuccess)
            e = cudaMemcpy(P->units, funits.data(), funits.size() * sizeof(FftUnit), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&P->counter, sizeof(unsigned));
        if (e == cudaSuccess && ws_per > 0) {
            P->qws_per = ws_per;
            e = cudaMalloc(&P->qws, (size_t)(2 * std::max(1, c->sms)) * (size_t)ws_per * sizeof(float2));
        }
        if (e == cudaSuccess && funits_pairs.size() != funits.size()) {
            P->nunits_alt = (int)funits_pairs.size();
            e = cudaMalloc(&P->units_alt, funits_pairs.size() * sizeof(FftUnit));
            if (e == cudaSuccess)
                e = cudaMemcpy(P->units_alt, funits_pairs.data(), funits_pairs.size() * sizeof(FftUnit),
                               cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess && !units.empty()) {
        P->nunits = (int)units.size();
        e = cudaMalloc(&P->units, units.size() * sizeof(CztUnit));
        if (e == cudaSuccess)
            e = cudaMemcpy(P->units, units.data(), units.size() * sizeof(CztUnit), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&P->counter, sizeof(unsigned));
        for (auto& kv : vkeys) {
            if (e != cudaSuccess) break;
            RaggedItem* dk = nullptr;
            e = cudaMalloc(&dk, kv.second.size() * sizeof(RaggedItem));
            if (e == cudaSuccess)
                e = cudaMemcpy(dk, kv.second.data(), kv.second.size() * sizeof(RaggedItem), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = czt_vpool_build(kv.first, dk, (int64_t)kv.second.size(), P->vpool, c->block_tw, P->cap);
            if (e == cudaSuccess) e = cudaStreamSynchronize(P->cap);
            if (dk) cudaFree(dk);
        }
    }
    if (e != cudaSuccess) return bail(ctx_cuda_fail(c, e, "ragged plan"));
    // ---- per-class tables ------------------------------------------------------
    for (RaggedClass& k : P->classes) {
        spec_status s = SPEC_OK;
        if (k.path == 0) s = ctx_plan_table(c, 0, k.fp, &k.tab);
        if (k.path == 3) s = ctx_plan_table(c, 1, k.fp, &k.tab);
        if (s != SPEC_OK) return bail(s);
        if (k.path == 1) {
            e = czt_ragged_tables(k.L, P->items + k.first, k.count, P->tables, tw_for(c, k.L), P->cap);
            if (e != cudaSuccess) return bail(ctx_cuda_fail(c, e, "ragged CZT tables"));
        }
    }
    e = cudaStreamSynchronize(P->cap);
    if (e != cudaSuccess) return bail(ctx_cuda_fail(c, e, "ragged plan"));
    // ---- autotune: the FFT queue's long traces as whole-trace workspace units
    //      or as residue-pair units, by timing the launch both ways -----------
    if (P->units_alt) {
        auto time_queue = [&](void* u, int nu) {
            cudaEvent_t ea, eb;
            cudaEventCreate(&ea);
            cudaEventCreate(&eb);
            float best = 1e30f;
            for (int r = 0; r < 4; ++r) {
                cudaEventRecord(ea, P->cap);
                cudaError_t le = cudaMemsetAsync(P->counter, 0, sizeof(unsigned), P->cap);
                if (le == cudaSuccess)
                    le = fft_queue_launch(P->items, (const FftUnit*)u, nu, P->counter, x, c->block_tw, X, P->qws,
                                          P->qws_per, 2 * std::max(1, c->sms), P->cap);
                cudaEventRecord(eb, P->cap);
                if (le != cudaSuccess || cudaEventSynchronize(eb) != cudaSuccess) {
                    best = 1e30f;
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ea, eb);
                if (r > 0) best = std::min(best, ms);
            }
            cudaEventDestroy(ea);
            cudaEventDestroy(eb);
            cudaGetLastError();
            return best;
        };
        const float t_ws = time_queue(P->units, P->nunits);
        const float t_pairs = time_queue(P->units_alt, P->nunits_alt);
        if (t_pairs < t_ws) {
            std::swap(P->units, P->units_alt);
            std::swap(P->nunits, P->nunits_alt);
        }
    }
    // ---- autotune: FFT classes choose lanes and pass radix by timing ----------
    for (RaggedClass& k : P->classes) {
        if (k.path != 0) continue;
        RaggedClass best = k;
        best.tuned_us = 1e30f;
        RaggedClass base = k;
        {
            // the cluster kernel (where it has an instance) is one more candidate
            RaggedClass cl = k;
            std::string why;
            if (fft_plan(k.count, 2 * (int64_t)k.fp.LZ, 2 * (int64_t)k.fp.H, &cl.fp, &why, true) && cl.fp.clustered &&
                ctx_plan_table(c, 0, cl.fp, &cl.tab) == SPEC_OK) {
                const float t = 1e3f * time_class(c, P, cl, x, taps, X);
                if (t < best.tuned_us) {
                    best = cl;
                    best.tuned_us = t;
                }
            }
        }
        for (int emax : {16, 32}) {
            if (emax == 32 && !(k.fp.LZ == 512 || k.fp.LZ == 1024 || k.fp.LZ == 8192)) continue;
            for (int lanes : {1, 2}) {
                RaggedClass cand = base;
                cand.fp.emax = emax;
                cand.fp.E = std::min(emax, cand.fp.LZ);
                cand.fp.T = cand.fp.LZ / cand.fp.E;
                if (emax == 32) cand.fp.dual = cand.fp.fixed = false;
                if (lanes == 2 && !cand.fp.dual) continue;
                cand.lanes = lanes;
                if (emax != base.fp.emax && ctx_plan_table(c, 0, cand.fp, &cand.tab) != SPEC_OK) continue;
                const float t = 1e3f * time_class(c, P, cand, x, taps, X);
                if (t < best.tuned_us) {
                    best = cand;
                    best.tuned_us = t;
                }
            }
        }
        if (best.tuned_us < 1e29f) k = best;
    }
    // ---- autotune: the work queue against the per-shape launches -------------
    P->use_queue = P->nunits > 0;
    if (P->nunits > 0) {
        auto time_graph = [&]() {
            if (capture(c, P, x, taps, X) != SPEC_OK) return 1e30f;
            cudaEvent_t ea, eb;
            cudaEventCreate(&ea);
            cudaEventCreate(&eb);
            float best = 1e30f;
            for (int r = 0; r < 4; ++r) {
                cudaEventRecord(ea, P->cap);
                cudaError_t le = cudaGraphLaunch(P->exec, P->cap);
                cudaEventRecord(eb, P->cap);
                if (le != cudaSuccess || cudaEventSynchronize(eb) != cudaSuccess) {
                    best = 1e30f;
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ea, eb);
                if (r > 0) best = std::min(best, ms);
            }
            cudaEventDestroy(ea);
            cudaEventDestroy(eb);
            cudaGetLastError();
            return best;
        };
        P->use_queue = false;
        const float t_classes = time_graph();
        P->use_queue = true;
        const float t_queue = time_graph();
        P->use_queue = c->ragged_queue >= 0 ? c->ragged_queue == 1 : t_queue <= t_classes;
        P->t_queue_us = 1e3f * t_queue;
        P->t_classes_us = 1e3f * t_classes;
        if (P->exec) {
            cudaGraphExecDestroy(P->exec);      // captured again for the chosen form by the caller
            P->exec = nullptr;
        }
    }
    *out = P;
    return SPEC_OK;
}

}  // namespace

extern "C" spec_status spec_ragged(spec_ctx* c, int kind, const spec_desc* descs, int64_t count, double fs,
                                   const float* x_pool, const float* taps_pool, float* X_pool, void* stream) {
    if (!c) return SPEC_EINVAL;
    if (kind != SPEC_KIND_FFT && kind != SPEC_KIND_CZT && kind != SPEC_KIND_ZOOM)
        return ctx_fail(c, SPEC_EINVAL, "unknown transform kind");
    if (count < 0 || (count > 0 && (!descs || !x_pool || !X_pool)))
        return ctx_fail(c, SPEC_EINVAL, "count must be >= 0 with descriptors and pools");
    if (count > (int64_t(1) << 31) - 1) return ctx_fail(c, SPEC_EINVAL, "count too large");
    if (!(fs > 0.0) || !std::isfinite(fs)) return ctx_fail(c, SPEC_EINVAL, "fs must be finite and > 0");
    if (kind == SPEC_KIND_ZOOM && count > 0 && !taps_pool) return ctx_fail(c, SPEC_EINVAL, "taps pool is NULL");
    if (count == 0) return SPEC_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    struct Restore {
        int d;
        ~Restore() {
            if (d >= 0) cudaSetDevice(d);
        }
    } restore{prev != c->device ? prev : -1};
    if (!ctx_is_device_ptr(x_pool) || !ctx_is_device_ptr(X_pool) ||
        (kind == SPEC_KIND_ZOOM && !ctx_is_device_ptr(taps_pool)))
        return ctx_fail(c, SPEC_EINVAL, "ragged pools must be device memory");
    float2* X = reinterpret_cast<float2*>(X_pool);
    RaggedPlan* P = nullptr;
    for (RaggedPlan* p : c->ragged)
        if (same_descs(p, kind, fs, descs, count)) P = p;
    if (!P) {
        // the plan's table builds and timing runs use their own stream: let
        // the caller's pending work on the pools finish first
        cudaError_t se = cudaStreamSynchronize((cudaStream_t)stream);
        if (se != cudaSuccess) return ctx_cuda_fail(c, se, "stream");
        spec_status s = build_plan(c, kind, descs, count, fs, x_pool, taps_pool, X, &P);
        if (s != SPEC_OK) return s;
        if (c->ragged.size() >= 8) {
            cudaDeviceSynchronize();
            ragged_plan_free(c->ragged.front());
            c->ragged.erase(c->ragged.begin());
        }
        c->ragged.push_back(P);
    }
    if (!P->exec || P->gx != x_pool || P->gt != taps_pool || P->gX != X) {
        spec_status s = capture(c, P, x_pool, taps_pool, X);
        if (s != SPEC_OK) return s;
    }
    cudaError_t e = cudaGraphLaunch(P->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return ctx_cuda_fail(c, e, "graph launch");
    return SPEC_OK;
}

// Kernel launches in one replay of the cached plan for these descriptors
// (the queue launch, one per remaining class, plus the FIR launch of the
// large Zoom path); -1 if the context holds no such plan.
extern "C" int64_t spec_ragged_launches(const spec_ctx* c, int kind, const spec_desc* descs, int64_t count,
                                        double fs) {
    if (!c || count < 0 || (count > 0 && !descs)) return -1;
    for (const RaggedPlan* p : c->ragged)
        if (same_descs(p, kind, fs, descs, count)) {
            int64_t n = (p->fir_count > 0 ? 1 : 0) + (p->use_queue ? 1 : 0);
            for (const RaggedClass& k : p->classes)
                if (k.path != 3 && !(p->use_queue && k.in_queue)) ++n;
            for (const RaggedClass& k : p->classes)
                if (k.path == 3) ++n;
            return n;
        }
    return -1;
}

// How the cached plan for these descriptors runs: 1 if its graph launches the
// persistent work queue (0: the per-shape launches), and the two forms' times
// measured when the plan was built (microseconds; 0 where there was no queue).
// -1 if the context holds no such plan.
extern "C" int spec_ragged_plan_info(const spec_ctx* c, int kind, const spec_desc* descs, int64_t count, double fs,
                                     float* t_queue_us, float* t_classes_us) {
    if (!c || count < 0 || (count > 0 && !descs)) return -1;
    for (const RaggedPlan* p : c->ragged)
        if (same_descs(p, kind, fs, descs, count)) {
            if (t_queue_us) *t_queue_us = p->t_queue_us;
            if (t_classes_us) *t_classes_us = p->t_classes_us;
            return p->use_queue ? 1 : 0;
        }
    return -1;
}
