// ctx.h -- the library context (opaque to callers of include/spec.h) and the
// helpers the API translation units share.  Internal.
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <initializer_list>
#include <map>
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
    int kind = 0;        // 0: padded real FFT tables, 1: pruned complex FFT tables, 2: multi-pass twiddles (H = period log2),
                         // 4: mixed-radix padded FFT tables
    int H = 0, LZ = 0, emax = 16;
    int layout = 0;      // kind 0: generic (0), fixed two-lane (1), cluster (2) or fused-unpack (3) table layout
    float2* tab = nullptr;
};

struct GemmZEntry {       // cached FP16 split of Z for the GEMM chirp-z
    int64_t n = 0, m = 0;
    uint64_t A = 0, B = 0;
    double a0 = 1.0, w0 = 1.0;           // contour radius parameters (1, 1: the unit circle)
    bool bf16 = false;                   // one BF16 part (SPEC_CZT_GEMM_BF16X1) instead of the FP16 split
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
    bool fft_cluster = false;            // SPEC_FFT_CLUSTER=1: long traces on k_fft_real_cluster
    std::string fft_variant;             // SPEC_FFT_VARIANT: pin a padded-FFT kernel variant by name
    bool gemm_fused = false;             // SPEC_GEMM_FUSED=1: FP16 split inside the tensor-core product
    int ragged_queue = -1;               // SPEC_RAGGED_QUEUE: 1 always / 0 never the work queue, -1 timed
    std::map<std::string, std::string> tune;   // SPEC_CZT_AUTO decisions ("czt n=.. m=.. b=.." -> mode)
    std::string tune_path, tune_device;        // SPEC_AUTOTUNE_CACHE file and this device's tag
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
// autotune.cu: the persisted decision cache and the SPEC_CZT_AUTO decision
bool tune_file_read(const std::string& path, const std::string& device, std::map<std::string, std::string>* entries);
bool tune_file_write(const std::string& path, const std::string& device,
                     const std::map<std::string, std::string>& entries);
bool tune_file_store(const std::string& path, const std::string& device, const std::string& key,
                     const std::string& value);
std::string device_tag(int device);
// the fastest of `names` for `key` (remembered, cached on file, or measured
// by `run(i)` on the caller's buffers); -1 with *status set on failure
int tune_pick(spec_ctx* c, const std::string& key, const std::vector<std::string>& names,
              const std::function<cudaError_t(int)>& run, cudaStream_t st, spec_status* status);
// "what v0:v1:..." -- the shape a variant decision belongs to
std::string tune_key(const char* what, std::initializer_list<long long> v);
spec_status czt_auto_decide(spec_ctx* c, int64_t batch, int64_t n, double fs, double f1, double f2, int64_t m,
                            int* mode, cudaStream_t st);
}  // namespace spec
