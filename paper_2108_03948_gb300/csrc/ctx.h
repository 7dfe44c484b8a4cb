// ctx.h -- the library context (opaque to callers of include/spec.h) and the
// helpers the API translation units share.  Internal.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "spec.h"
#include "spec_internal.h"

struct CztEntry {
    spec::CztTables t;
    bool multipass = false;              // multi-pass Bluestein (L above one CTA)
    spec::LongPlan lp;
    float2* tw2 = nullptr;               // its twiddle table (inside mem)
    void* mem = nullptr;
    cudaEvent_t ready = nullptr;
    uint64_t last_use = 0;
};

struct FftEntry {
    int kind = 0;        // 0: padded real FFT tables, 1: pruned complex FFT tables, 2: multi-pass twiddles (H = period log2)
    int H = 0, LZ = 0, emax = 16;
    bool fixed = false;  // kind 0 with the packed tables of the fixed two-lane kernel
    float2* tab = nullptr;
};

struct GemmZEntry {       // cached FP16 split of Z for the GEMM chirp-z
    int64_t n = 0, m = 0;
    uint64_t A = 0, B = 0;
    double a0 = 1.0, w0 = 1.0;           // contour radius parameters (1, 1: the unit circle)
    int* col_pow = nullptr;              // off the circle: per-bin column exponents (inside z)
    void* z = nullptr;
    cudaEvent_t ready = nullptr;
    uint64_t last_use = 0;
};

struct RaggedPlan;       // ragged.cu
void ragged_plan_free(RaggedPlan* p);

struct spec_ctx {
    int device = 0;
    std::string err;
    float2* block_tw = nullptr;          // BlockFFT twiddles of every size
    int lanes = 0;                       // 0: per transform (two packed lanes for the padded FFT, one for the
                                         // chirp-z and Zoom: measured fastest); 1 or 2: forced everywhere
    std::vector<FftEntry> fft;
    std::vector<CztEntry> czt;
    std::vector<GemmZEntry> gemm_z;
    unsigned* status = nullptr;          // device word: bit 0 = a bounded wait gave up
    int sms = 0;                         // multiprocessors (persistent grids)
    uint64_t wait_timeout_ns = 1000000000ull;
    std::vector<RaggedPlan*> ragged;     // cached ragged-batch plans (graph + per-trace tables)
    uint64_t tick = 0;
    void* stage[4] = {nullptr, nullptr, nullptr, nullptr};   // x, X (two host-buffer chunks each), taps, workspace
    size_t stage_bytes[4] = {0, 0, 0, 0};
    cudaStream_t copy[2] = {nullptr, nullptr};  // host-buffer uploads, downloads (created on first use)
    cudaEvent_t ev_in[2] = {nullptr, nullptr};   // per staging slot: upload done,
    cudaEvent_t ev_tr[2] = {nullptr, nullptr};   // transform done,
    cudaEvent_t ev_out[2] = {nullptr, nullptr};  // download done
};

namespace spec {
spec_status ctx_fail(spec_ctx* c, spec_status s, const std::string& why);
spec_status ctx_cuda_fail(spec_ctx* c, cudaError_t e, const char* what);
bool ctx_is_device_ptr(const void* p);
// Cached per-shape twiddle tables: kind 0 padded real FFT, kind 1 pruned complex FFT.
spec_status ctx_plan_table(spec_ctx* c, int kind, const FftPlan& p, const float2** tab);
}  // namespace spec
