// ragged.cu -- spec_ragged: many traces that each bring their own length,
// band, point count, decimation and taps, transformed in one call.
//
// The first call with a given descriptor list builds a plan and caches it in
// the context:
//   * every descriptor is validated exactly as the single-shape entry point
//     would validate it (Section 2.1-2.3 conventions, include/spec.h);
//   * traces are grouped into classes by kernel instantiation (FFT: residue
//     length and H; CZT: Bluestein length L; Zoom: K, or (K, pruned length)
//     for the large path), and a device array of per-trace placements and
//     parameters (RaggedItem) is uploaded;
//   * CZT traces get their own chirp tables and kernel spectrum (float64
//     phases), built once on the device;
//   * an autotuner times the kernel variants a class admits (FFT: one or two
//     residues per thread, radix 16 or 32 passes) on the class's own traces
//     and keeps the fastest;
//   * one CUDA graph is captured with one launch per class, the classes on
//     parallel branches, so the whole batch is one graph launch.
// Later calls with the same descriptors replay the graph (re-captured if the
// pool pointers change).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
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
    size_t smem = 0;     // Zoom one-CTA: the largest need in the class
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
    delete p;
}

namespace {

bool same_descs(const RaggedPlan* p, int kind, double fs, const spec_desc* d, int64_t count) {
    return p->kind == kind && p->fs == fs && (int64_t)p->descs.size() == count &&
           (count == 0 || std::memcmp(p->descs.data(), d, (size_t)count * sizeof(spec_desc)) == 0);
}

const float2* tw_for(spec_ctx* c, int LF, int emax = 16) { return c->block_tw + block_twiddle_offset(LF, emax); }

cudaError_t launch_class(spec_ctx* c, RaggedPlan* P, const RaggedClass& k, cudaStream_t s, const float* x,
                         const float* taps, float2* X) {
    const RaggedItem* it = P->items + k.first;
    switch (k.path) {
        case 0:
            return fft_launch(k.fp, x, k.count, 0, 0, tw_for(c, k.fp.LZ, k.fp.emax), k.tab, X, 0, s, k.lanes, it);
        case 1:
            return czt_ragged_launch(k.L, it, k.count, x, P->tables, tw_for(c, k.L), X, s);
        case 2:
            return zoom_ragged_launch(k.K, it, k.count, k.smem, x, taps, tw_for(c, k.K), X, s);
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
    size_t br = 0;
    // one branch per class of paths 0-2; the large Zoom path (FIR, then its
    // pruned-FFT classes) forms one more branch
    for (const RaggedClass& k : P->classes) {
        if (k.path == 3 || le != cudaSuccess) continue;
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
    int64_t tab_total = 0, work_total = 0;
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
    if (e == cudaSuccess && work_total > 0) e = cudaMalloc(&P->work, (size_t)work_total * sizeof(float2));
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
    // ---- autotune: FFT classes choose lanes and pass radix by timing ----------
    for (RaggedClass& k : P->classes) {
        if (k.path != 0) continue;
        RaggedClass best = k;
        best.tuned_us = 1e30f;
        for (int emax : {16, 32}) {
            if (emax == 32 && !(k.fp.LZ == 512 || k.fp.LZ == 1024 || k.fp.LZ == 8192)) continue;
            for (int lanes : {1, 2}) {
                RaggedClass cand = k;
                cand.fp.emax = emax;
                cand.fp.E = std::min(emax, cand.fp.LZ);
                cand.fp.T = cand.fp.LZ / cand.fp.E;
                if (emax == 32) cand.fp.dual = cand.fp.fixed = false;
                if (lanes == 2 && !cand.fp.dual) continue;
                cand.lanes = lanes;
                if (emax != k.fp.emax && ctx_plan_table(c, 0, cand.fp, &cand.tab) != SPEC_OK) continue;
                const float t = 1e3f * time_class(c, P, cand, x, taps, X);
                if (t < best.tuned_us) {
                    best = cand;
                    best.tuned_us = t;
                }
            }
        }
        if (best.tuned_us < 1e29f) k = best;
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
// (one per class, plus the FIR launch of the large Zoom path); -1 if the
// context holds no such plan.
extern "C" int64_t spec_ragged_launches(const spec_ctx* c, int kind, const spec_desc* descs, int64_t count,
                                        double fs) {
    if (!c || count < 0 || (count > 0 && !descs)) return -1;
    for (const RaggedPlan* p : c->ragged)
        if (same_descs(p, kind, fs, descs, count)) return (int64_t)p->classes.size() + (p->fir_count > 0 ? 1 : 0);
    return -1;
}
