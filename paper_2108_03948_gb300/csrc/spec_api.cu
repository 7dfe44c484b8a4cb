// spec_api.cu -- the C-ABI declared in include/spec.h: context, argument
// validation (before any launch), host-buffer staging, the Bluestein table
// cache, and dispatch to the kernels.  No exception crosses the boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "ctx.h"
#include "fft_block.cuh"
#include "spec.h"
#include "spec_internal.h"

namespace spec {

static int block_twiddle_total16() { return fft_twiddle_offset(kMaxBlockFFT) + fft_twiddle_entries(kMaxBlockFFT); }
int block_twiddle_total() {
    return block_twiddle_total16() + fft_twiddle_offset(kMaxBlockFFT, 32) + fft_twiddle_entries(kMaxBlockFFT, 32);
}
int block_twiddle_offset(int LF, int emax) {
    if (emax == 32) return LF <= 32 ? 0 : block_twiddle_total16() + fft_twiddle_offset(LF, 32);
    return LF <= 16 ? 0 : fft_twiddle_offset(LF);
}

// Twiddles of the Stockham passes of every BlockFFT size (the layout of
// FFTShape::tw_off): pass p >= 1 of radix R after NS points holds
// e^{-j 2 pi r k/(NS R)} at [NS - EMAX + (r-1) NS + k].  float64, exact
// argument reduction, rounded to float.
static void fill_emax(float2* host, int emax) {
    const double two_pi = 6.283185307179586476925286766559;
    const int le = ilog2(emax);
    for (int LF = 2 * emax; LF <= kMaxBlockFFT; LF <<= 1) {
        float2* o = host + block_twiddle_offset(LF, emax);
        const int lg = ilog2(LF), npb = lg / le, rem = 1 << (lg % le);
        const int npass = npb + (rem > 1 ? 1 : 0);
        int ns = 1;
        for (int p = 0; p < npass; ++p) {
            const int R = p < npb ? emax : rem;
            if (p >= 1)
                for (int r = 1; r < R; ++r)
                    for (int k = 0; k < ns; ++k) {
                        const int64_t S = (int64_t)ns * R;
                        const double ang = two_pi * (double)(((int64_t)r * k) % S) / (double)S;
                        o[ns - emax + (r - 1) * ns + k] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
                    }
            ns *= R;
        }
    }
}

void block_twiddle_fill(float2* host) {
    fill_emax(host, 16);
    fill_emax(host, 32);
}

uint64_t cycles_to_fixed(double cycles) {
    double fr = cycles - std::floor(cycles);           // [0, 1)
    double v = std::ldexp(fr, 64);
    if (!(v < 18446744073709551616.0)) v = 0.0;        // fr rounded up to 1
    return (uint64_t)v;
}

}  // namespace spec

using namespace spec;

static std::string g_create_err;
static const size_t kCztCacheMax = 64;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

spec_status fail(spec_ctx* c, spec_status s, const std::string& why) {
    c->err = why;
    return s;
}

spec_status cuda_fail(spec_ctx* c, cudaError_t e, const char* what) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SPEC_ENOMEM : SPEC_ECUDA;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + nb && pb < pa + na;
}

bool is_finite(double v) { return std::isfinite(v); }

// Staging slots grow only; a buffer being replaced may still be in use by
// work queued on any stream, so the device drains first.
spec_status ensure_stage(spec_ctx* c, int slot, size_t bytes) {
    if (c->stage_bytes[slot] >= bytes) return SPEC_OK;
    if (c->stage[slot]) {
        cudaDeviceSynchronize();
        cudaFree(c->stage[slot]);
    }
    c->stage[slot] = nullptr;
    c->stage_bytes[slot] = 0;
    cudaError_t e = cudaMalloc(&c->stage[slot], bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "staging buffer");
    c->stage_bytes[slot] = bytes;
    return SPEC_OK;
}

// Host buffers.  A call whose x or X is host memory runs the batch in chunks
// of traces through two device staging slots per direction, so that the
// upload of chunk i+1 (copy stream 0), the transform of chunk i (the caller's
// stream) and the download of chunk i-1 (copy stream 1) overlap.  Events
// order the reuse of the slots:
//   upload i     waits for transform i-2 (which read its input slot),
//   transform i  waits for upload i and for download i-2 (its output slot),
//   download i   waits for transform i.
// The call returns once X holds the result, so the caller may reuse the host
// buffers at once.  `fn` runs the transform of one chunk on device pointers.
using ChunkFn = std::function<spec_status(const float* xd, int64_t ld_xd, float2* Xd, int64_t ld_Xd, int64_t nb)>;

// Traces per chunk: one chunk below 16 MiB of host traffic; otherwise 4 - 64
// chunks of about 32 MiB each, rounded up to a multiple of 64 traces.  No
// chunk holds a single trace unless the batch does (the two-trace kernels
// then see the same pairs as in a device-pointer call).
int64_t pipeline_chunk(int64_t batch, int64_t bytes_per_trace) {
    const double total = (double)batch * (double)bytes_per_trace;
    if (total < 16.0 * 1048576.0) return std::max<int64_t>(1, batch);
    const int64_t parts = (int64_t)std::min(64.0, std::max(4.0, total / (32.0 * 1048576.0)));
    int64_t chunk = (batch + parts - 1) / parts;
    if (chunk > 64) chunk = (chunk + 63) / 64 * 64;
    while (chunk < batch && batch % chunk == 1) chunk += 2;
    return std::max<int64_t>(1, std::min(chunk, batch));
}

spec_status ensure_copy_streams(spec_ctx* c) {
    if (c->copy[0]) return SPEC_OK;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&c->copy[k], cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&c->ev_in[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_tr[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "copy streams");
    return SPEC_OK;
}

spec_status host_pipeline(spec_ctx* c, const float* x, int64_t batch, int64_t n, int64_t ld_x, float* X,
                          int64_t bins, int64_t ld_X, cudaStream_t st, const ChunkFn& fn) {
    const bool xh = !is_device_ptr(x), Xh = !is_device_ptr(X);
    const int64_t chunk = pipeline_chunk(batch, (xh ? n * 4 : 0) + (Xh ? bins * 8 : 0));
    spec_status s = SPEC_OK;
    if ((s = ensure_copy_streams(c)) != SPEC_OK) return s;
    if (xh && (s = ensure_stage(c, 0, 2 * (size_t)chunk * (size_t)n * sizeof(float))) != SPEC_OK) return s;
    if (Xh && (s = ensure_stage(c, 1, 2 * (size_t)chunk * (size_t)bins * sizeof(float2))) != SPEC_OK) return s;
    cudaStream_t up = c->copy[0], down = c->copy[1];
    float2* X2 = reinterpret_cast<float2*>(X);
    const int64_t nch = (batch + chunk - 1) / chunk;
    cudaError_t e = cudaSuccess;
    auto download = [&](int64_t i) {
        const int sl = (int)(i & 1);
        const int64_t b0 = i * chunk, nb = std::min(chunk, batch - b0);
        e = cudaStreamWaitEvent(down, c->ev_tr[sl], 0);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(X2 + b0 * ld_X, ld_X * sizeof(float2), (float2*)c->stage[1] + sl * chunk * bins,
                                  bins * sizeof(float2), bins * sizeof(float2), nb, cudaMemcpyDeviceToHost, down);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_out[sl], down);
    };
    for (int64_t i = 0; i < nch; ++i) {
        const int sl = (int)(i & 1);
        const int64_t b0 = i * chunk, nb = std::min(chunk, batch - b0);
        const float* xd = x + b0 * ld_x;
        int64_t ld_xd = ld_x;
        if (xh) {
            float* slot = (float*)c->stage[0] + sl * chunk * n;
            e = cudaStreamWaitEvent(up, c->ev_tr[sl], 0);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(slot, n * sizeof(float), xd, ld_x * sizeof(float), n * sizeof(float), nb,
                                      cudaMemcpyHostToDevice, up);
            if (e == cudaSuccess) e = cudaEventRecord(c->ev_in[sl], up);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->ev_in[sl], 0);
            xd = slot;
            ld_xd = n;
        }
        float2* Xd = X2 + b0 * ld_X;
        int64_t ld_Xd = ld_X;
        if (Xh) {
            Xd = (float2*)c->stage[1] + sl * chunk * bins;
            ld_Xd = bins;
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->ev_out[sl], 0);
        }
        if (e != cudaSuccess) break;
        if ((s = fn(xd, ld_xd, Xd, ld_Xd, nb)) != SPEC_OK) break;
        if ((e = cudaEventRecord(c->ev_tr[sl], st)) != cudaSuccess) break;
        if (Xh && i > 0) download(i - 1);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess && s == SPEC_OK && Xh) {
        download(nch - 1);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->ev_out[(nch - 1) & 1], 0);
    }
    // whatever happened, nothing may still be copying from or to the
    // caller's buffers when the call returns
    const cudaError_t e1 = cudaStreamSynchronize(up), e2 = cudaStreamSynchronize(down);
    const cudaError_t e3 = cudaStreamSynchronize(st);
    if (s != SPEC_OK) return s;
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3;
    if (e != cudaSuccess) return cuda_fail(c, e, "host-buffer transform");
    return SPEC_OK;
}

spec_status check_common(spec_ctx* c, const float* x, int64_t batch, int64_t n, int64_t ld_x,
                         double fs, const float* X, int64_t bins, int64_t ld_X) {
    if (!x || !X) return fail(c, SPEC_EINVAL, "x and X must not be NULL");
    if (batch < 0) return fail(c, SPEC_EINVAL, "batch must be >= 0");
    if (n < 1 || n > (int64_t(1) << 24)) return fail(c, SPEC_EINVAL, "n must be in [1, 2^24]");
    if (ld_x < n) return fail(c, SPEC_EINVAL, "ld_x must be >= n");
    if (ld_X < bins) return fail(c, SPEC_EINVAL, "ld_X must be >= the number of output bins");
    if (!(fs > 0.0) || !is_finite(fs)) return fail(c, SPEC_EINVAL, "fs must be finite and > 0");
    if (batch > 0) {
        const size_t bx = (size_t)((batch - 1) * ld_x + n) * sizeof(float);
        const size_t bX = (size_t)((batch - 1) * ld_X + bins) * sizeof(float2);
        if (overlaps(x, bx, X, bX)) return fail(c, SPEC_EINVAL, "x and X overlap");
    }
    return SPEC_OK;
}

int table_layout(int kind, const FftPlan& p) {
    if (kind != 0) return 0;
    return p.clustered ? 2 : p.fused ? (p.fold == 2 ? 4 : 3) : p.fixed ? 1 : 0;
}

// Per-shape twiddle tables of the padded real FFT (kind 0) and of the pruned
// complex FFT (kind 1), built on the host in float64 and cached.
spec_status plan_table(spec_ctx* c, int kind, const FftPlan& p, const float2** tab) {
    for (auto& it : c->fft)
        if (it.kind == kind && it.H == p.H && it.LZ == p.LZ && it.emax == p.emax && it.layout == table_layout(kind, p)) {
            *tab = it.tab;
            return SPEC_OK;
        }
    FftEntry ne;
    ne.kind = kind;
    ne.H = p.H;
    ne.LZ = p.LZ;
    ne.emax = p.emax;
    ne.layout = table_layout(kind, p);
    std::vector<float2> host((size_t)(kind == 0 ? fft_table_entries(p) : c2c_table_entries(p)));
    if (kind == 0) fft_fill_table(p, host.data());
    else c2c_fill_table(p, host.data());
    cudaError_t e = cudaMalloc(&ne.tab, host.size() * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(ne.tab, host.data(), host.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (ne.tab) cudaFree(ne.tab);
        return cuda_fail(c, e, "FFT tables");
    }
    c->fft.push_back(ne);
    *tab = ne.tab;
    return SPEC_OK;
}

// Chirp-z as the tensor-core product x Z^T (k_gemm.cu): Z cached per
// (N, M, f1/fs, step/fs), the batch run in chunks whose FP16 split fits a
// ~1 GiB workspace.
spec_status czt_gemm(spec_ctx* c, const float* x, int64_t batch, int64_t n, int64_t ld_x, double fs, double f1,
                     double f2, int64_t m, int terms, float* X, int64_t ld_X, cudaStream_t st, double a0 = 1.0,
                     double w0 = 1.0) {
    if (gemm_z_bytes(n, m) > (size_t(1) << 31))
        return fail(c, SPEC_EUNSUPPORTED, "GEMM chirp-z: Z above 2 GiB (use SPEC_CZT_BLUESTEIN)");
    // off the unit circle: column k of Z is scaled by 2^-e_k, e_k the exponent
    // of its largest magnitude max(1, exp((N-1)(-ln a0 + k ln w0)))
    const bool spiral = a0 != 1.0 || w0 != 1.0;
    std::vector<int> col_pow;
    if (spiral) {
        col_pow.resize((size_t)m);
        const double la = std::log(a0), lw = std::log(w0);
        for (int64_t k = 0; k < m; ++k) {
            const double lg = (double)(n - 1) * (-la + (double)k * lw) / 0.6931471805599453;
            if (lg > 100.0)
                return fail(c, SPEC_EUNSUPPORTED, "spiral chirp-z: the contour's |z_k|^-n exceeds 2^100");
            col_pow[(size_t)k] = lg > 0.0 ? (int)std::ceil(lg) : 0;
        }
    }
    if (batch == 0) return SPEC_OK;
    DeviceGuard g(c->device);
    const double step = m > 1 ? (f2 - f1) / (double)(m - 1) : 0.0;
    const uint64_t A = cycles_to_fixed(f1 / fs);
    const uint64_t B = cycles_to_fixed(step / fs);
    GemmZEntry* en = nullptr;
    const bool bf16 = terms < 0;
    for (auto& it : c->gemm_z)
        if (it.n == n && it.m == m && it.A == A && it.B == B && it.a0 == a0 && it.w0 == w0 && it.bf16 == bf16) en = &it;
    if (!en) {
        if (c->gemm_z.size() >= kCztCacheMax) {
            auto lru = std::min_element(c->gemm_z.begin(), c->gemm_z.end(),
                                        [](const GemmZEntry& a, const GemmZEntry& b) { return a.last_use < b.last_use; });
            cudaDeviceSynchronize();
            cudaFree(lru->z);
            cudaEventDestroy(lru->ready);
            c->gemm_z.erase(lru);
        }
        GemmZEntry ne;
        ne.n = n; ne.m = m; ne.A = A; ne.B = B; ne.a0 = a0; ne.w0 = w0; ne.bf16 = bf16;
        const size_t zb = (gemm_z_bytes(n, m) + 255) / 256 * 256;
        cudaError_t e = cudaMalloc(&ne.z, zb + (spiral ? (size_t)m * sizeof(int) : 0));
        if (e != cudaSuccess) return cuda_fail(c, e, "GEMM Z table");
        e = cudaEventCreateWithFlags(&ne.ready, cudaEventDisableTiming);
        if (e != cudaSuccess) { cudaFree(ne.z); return cuda_fail(c, e, "event"); }
        if (spiral) {
            ne.col_pow = (int*)((uint8_t*)ne.z + zb);
            e = cudaMemcpy(ne.col_pow, col_pow.data(), (size_t)m * sizeof(int), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess)
            e = spiral ? gemm_build_z_spiral(n, m, A, B, std::log(a0), std::log(w0), ne.col_pow, ne.z, st)
                       : gemm_build_z(n, m, A, B, ne.z, st, bf16);
        if (e == cudaSuccess) e = cudaEventRecord(ne.ready, st);
        if (e != cudaSuccess) {
            cudaFree(ne.z);
            cudaEventDestroy(ne.ready);
            return cuda_fail(c, e, "GEMM Z build");
        }
        c->gemm_z.push_back(ne);
        en = &c->gemm_z.back();
    } else {
        cudaError_t e = cudaStreamWaitEvent(st, en->ready, 0);
        if (e != cudaSuccess) return cuda_fail(c, e, "table wait");
    }
    en->last_use = ++c->tick;
    spec_status s;
    float2* X2 = reinterpret_cast<float2*>(X);
    // The FP16 split then the product, in chunks only when the workspace
    // would exceed 512 MiB (one product over the whole batch keeps the tile
    // waves full; smaller products measured slower, even with the split of
    // the next chunk overlapped).
    const int64_t per_row = (int64_t)gemm_padded_n(n) * 4 + 4;
    int64_t chunk = std::max<int64_t>(128, ((int64_t(1) << 29) / per_row) / 128 * 128);
    chunk = std::min(chunk, batch);
    if ((s = ensure_stage(c, 3, gemm_work_bytes(chunk, n))) != SPEC_OK) return s;
    for (int64_t b0 = 0; b0 < batch; b0 += chunk) {
        const int64_t nb = std::min(chunk, batch - b0);
        // the FP16 split as a pass of its own, then the product; with
        // SPEC_GEMM_FUSED=1 the split runs inside the product instead (FP32
        // boxes of x by TMA, converter warps; only the row exponents are a
        // pass), measured slower on GB300 and therefore not the default
        const float* xb = x + b0 * ld_x;
        const bool fused = c->gemm_fused && gemm_fused_ok(xb, ld_x);
        cudaError_t e = fused ? gemm_rowpow_launch(xb, nb, n, ld_x, c->stage[3], st)
                              : gemm_split_launch(xb, nb, n, ld_x, terms, c->stage[3], st);
        if (e == cudaSuccess)
            e = gemm_mul_launch(nb, n, m, terms, en->z, c->stage[3], X2 + b0 * ld_X, ld_X, c->status, c->sms,
                                c->wait_timeout_ns, st, en->col_pow, fused ? xb : nullptr, ld_x);
        if (e != cudaSuccess) return cuda_fail(c, e, "GEMM chirp-z launch");
    }
    return SPEC_OK;
}

// Twiddle table of the multi-pass transforms (period 2^logTw), cached.
spec_status long_table(spec_ctx* c, const LongPlan& p, const float2** tab) {
    for (auto& it : c->fft)
        if (it.kind == 2 && it.H == p.logTw) {
            *tab = it.tab;
            return SPEC_OK;
        }
    FftEntry ne;
    ne.kind = 2;
    ne.H = p.logTw;
    std::vector<float2> host((size_t)long_fft_table_entries(p));
    long_fill_tw(p, host.data());
    cudaError_t e = cudaMalloc(&ne.tab, host.size() * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(ne.tab, host.data(), host.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (ne.tab) cudaFree(ne.tab);
        return cuda_fail(c, e, "multi-pass twiddles");
    }
    c->fft.push_back(ne);
    *tab = ne.tab;
    return SPEC_OK;
}

// Workspace of the multi-pass transforms: whole traces, at most ~1 GiB and
// 65535 traces per chunk.
spec_status long_work(spec_ctx* c, const LongPlan& p, int64_t batch, float2** work, int64_t* traces) {
    const int64_t per = p.work_per_trace * (int64_t)sizeof(float2);
    int64_t t = std::max<int64_t>(1, (int64_t(1) << 30) / per);
    t = std::min<int64_t>({t, batch, 65535});
    spec_status s = ensure_stage(c, 3, (size_t)(t * per));
    if (s != SPEC_OK) return s;
    *work = (float2*)c->stage[3];
    *traces = t;
    return SPEC_OK;
}

}  // namespace

namespace spec {
spec_status ctx_fail(spec_ctx* c, spec_status s, const std::string& why) { return fail(c, s, why); }
spec_status ctx_cuda_fail(spec_ctx* c, cudaError_t e, const char* what) { return cuda_fail(c, e, what); }
bool ctx_is_device_ptr(const void* p) { return is_device_ptr(p); }
spec_status ctx_plan_table(spec_ctx* c, int kind, const FftPlan& p, const float2** tab) {
    return plan_table(c, kind, p, tab);
}
}  // namespace spec

extern "C" {

spec_status spec_ctx_create(spec_ctx** ctx, int device) {
    if (!ctx) {
        g_create_err = "ctx out-pointer is NULL";
        return SPEC_EINVAL;
    }
    *ctx = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_create_err = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return SPEC_ECUDA;
    }
    if (device < 0 || device >= count) {
        g_create_err = "device index out of range";
        return SPEC_EINVAL;
    }
    DeviceGuard g(device);
    e = cudaFree(nullptr);   // create the primary context now
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_create_err = std::string("cannot use device: ") + cudaGetErrorString(e);
        return SPEC_ECUDA;
    }
    spec_ctx* c = new (std::nothrow) spec_ctx();
    if (!c) {
        g_create_err = "out of host memory";
        return SPEC_ENOMEM;
    }
    c->device = device;
    if (const char* ev = std::getenv("SPEC_LANES")) c->lanes = std::atoi(ev);
    if (const char* ev = std::getenv("SPEC_FFT_CLUSTER")) c->fft_cluster = std::atoi(ev) == 1;
    if (const char* ev = std::getenv("SPEC_FFT_VARIANT")) c->fft_variant = ev;
    if (const char* ev = std::getenv("SPEC_GEMM_FUSED")) c->gemm_fused = std::atoi(ev) == 1;
    if (const char* ev = std::getenv("SPEC_RAGGED_QUEUE")) c->ragged_queue = std::atoi(ev) == 1 ? 1 : 0;
    c->tune_device = device_tag(device);
    if (const char* ev = std::getenv("SPEC_AUTOTUNE_CACHE")) {
        c->tune_path = ev;
        if (!c->tune_path.empty()) tune_file_read(c->tune_path, c->tune_device, &c->tune);
    }
    {
        std::vector<float2> host((size_t)block_twiddle_total());
        block_twiddle_fill(host.data());
        e = cudaMalloc(&c->block_tw, host.size() * sizeof(float2));
        if (e == cudaSuccess)
            e = cudaMemcpy(c->block_tw, host.data(), host.size() * sizeof(float2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g_create_err = std::string("twiddle tables: ") + cudaGetErrorString(e);
            if (c->block_tw) cudaFree(c->block_tw);
            delete c;
            return e == cudaErrorMemoryAllocation ? SPEC_ENOMEM : SPEC_ECUDA;
        }
    }
    e = cudaMalloc(&c->status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_create_err = std::string("status word: ") + cudaGetErrorString(e);
        if (c->status) cudaFree(c->status);
        cudaFree(c->block_tw);
        delete c;
        return SPEC_ECUDA;
    }
    if (const char* ev = std::getenv("SPEC_WAIT_TIMEOUT_MS")) {
        const long long ms = std::atoll(ev);
        if (ms > 0) c->wait_timeout_ns = (uint64_t)ms * 1000000ull;
    }
    *ctx = c;
    return SPEC_OK;
}

void spec_ctx_destroy(spec_ctx* c) {
    if (!c) return;
    {
        DeviceGuard g(c->device);
        cudaDeviceSynchronize();
        for (auto& en : c->czt) {
            if (en.mem) cudaFree(en.mem);
            if (en.ready) cudaEventDestroy(en.ready);
        }
        for (auto& en : c->fft)
            if (en.tab) cudaFree(en.tab);
        for (auto& en : c->gemm_z) {
            if (en.z) cudaFree(en.z);
            if (en.ready) cudaEventDestroy(en.ready);
        }
        if (c->status) cudaFree(c->status);
        for (RaggedPlan* rp : c->ragged) ragged_plan_free(rp);
        if (c->block_tw) cudaFree(c->block_tw);
        for (int i = 0; i < 4; ++i)
            if (c->stage[i]) cudaFree(c->stage[i]);
        for (int k = 0; k < 2; ++k) {
            if (c->copy[k]) cudaStreamDestroy(c->copy[k]);
            if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
            if (c->ev_tr[k]) cudaEventDestroy(c->ev_tr[k]);
            if (c->ev_out[k]) cudaEventDestroy(c->ev_out[k]);
        }
        cudaGetLastError();
    }
    delete c;
}

const char* spec_last_error(const spec_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

spec_status spec_ctx_check(spec_ctx* c, void* stream) {
    if (!c) return SPEC_EINVAL;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream");
    unsigned word = 0;
    e = cudaMemcpy(&word, c->status, sizeof(word), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "status word");
    if (word != 0) {
        e = cudaMemset(c->status, 0, sizeof(unsigned));
        if (e != cudaSuccess) return cuda_fail(c, e, "status word");
        return fail(c, SPEC_ETIMEOUT, "a bounded device-side wait gave up; the output of that call is incomplete");
    }
    c->err.clear();
    return SPEC_OK;
}

spec_status spec_selftest_wait_timeout(spec_ctx* c, int64_t timeout_us, void* stream) {
    if (!c) return SPEC_EINVAL;
    if (timeout_us < 1 || timeout_us > 1000000) return fail(c, SPEC_EINVAL, "timeout_us must be in [1, 10^6]");
    DeviceGuard g(c->device);
    cudaError_t e = wait_selftest_launch(c->status, (uint64_t)timeout_us * 1000ull, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "self-test launch");
    return SPEC_OK;
}

spec_status spec_fft(spec_ctx* c, const float* x, int64_t batch, int64_t n, int64_t ld_x, double fs,
                     int64_t n_fft, float* X, int64_t ld_X, void* stream) {
    if (!c) return SPEC_EINVAL;
    if (n_fft < 1 || n_fft > (int64_t(1) << 24))
        return fail(c, SPEC_EINVAL, "n_fft must be in [1, 2^24]");
    const int64_t bins = n_fft / 2 + 1;
    spec_status s = check_common(c, x, batch, n, ld_x, fs, X, bins, ld_X);
    if (s != SPEC_OK) return s;
    if (n_fft < n) return fail(c, SPEC_EINVAL, "n_fft must be >= n (padding never truncates)");
    MixedPlan mp;
    std::string why_mixed;
    if (!is_pow2(n_fft) && mixed_plan(n, n_fft, &mp, &why_mixed)) {
        // N_FFT with the factors 2, 3, 5, 7 only: the mixed-radix padded FFT
        if (batch == 0) return SPEC_OK;
        DeviceGuard g(c->device);
        cudaStream_t st = (cudaStream_t)stream;
        if (!is_device_ptr(x) || !is_device_ptr(X))
            return host_pipeline(c, x, batch, n, ld_x, X, bins, ld_X, st,
                                 [&](const float* xd, int64_t ld_xd, float2* Xd, int64_t ld_Xd, int64_t nb) {
                                     return spec_fft(c, xd, nb, n, ld_xd, fs, n_fft, (float*)Xd, ld_Xd, stream);
                                 });
        const float2* tab = nullptr;
        for (auto& it : c->fft)
            if (it.kind == 4 && it.H == mp.H && it.LZ == mp.LZ) tab = it.tab;
        if (!tab) {
            FftEntry ne;
            ne.kind = 4;
            ne.H = mp.H;
            ne.LZ = mp.LZ;
            std::vector<float2> host((size_t)mp.entries);
            mixed_fill_table(mp, host.data());
            cudaError_t e = cudaMalloc(&ne.tab, host.size() * sizeof(float2));
            if (e == cudaSuccess)
                e = cudaMemcpy(ne.tab, host.data(), host.size() * sizeof(float2), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                if (ne.tab) cudaFree(ne.tab);
                return cuda_fail(c, e, "mixed-radix FFT tables");
            }
            c->fft.push_back(ne);
            tab = ne.tab;
        }
        // the mixed-radix kernel or the chirp-z on the DFT grid, whichever
        // measures faster for this shape (SPEC_FFT_VARIANT pins one)
        spec_status sc = SPEC_OK;
        auto run = [&](int i) {
            if (i == 0) return mixed_launch(mp, x, batch, (int)n, ld_x, tab, reinterpret_cast<float2*>(X), ld_X, st);
            sc = spec_czt(c, x, batch, n, ld_x, fs, 0.0, fs * (double)(bins - 1) / (double)n_fft, bins,
                          SPEC_CZT_AUTO, X, ld_X, stream);
            return sc == SPEC_OK ? cudaSuccess : cudaErrorUnknown;
        };
        const std::vector<std::string> names{"mixed", "dftczt"};
        int pick = -1;
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == c->fft_variant) pick = (int)i;
        if (pick < 0) {
            pick = tune_pick(c, tune_key("fftmixed", {n_fft, mp.LZ}), names, run, st, &s);
            if (pick < 0) return s == SPEC_OK ? fail(c, SPEC_ECUDA, "spec_fft variant timing") : s;
        }
        cudaError_t e = run(pick);
        if (pick == 1 && sc != SPEC_OK) return sc;
        if (e != cudaSuccess) return cuda_fail(c, e, "spec_fft mixed-radix launch");
        return SPEC_OK;
    }
    if (!is_pow2(n_fft)) {
        // any other length: the same bins k fs/N_FFT, k = 0 .. N_FFT/2, as a
        // chirp-z with f1 = 0 and step fs/N_FFT (Eq. 11 on the DFT grid)
        return spec_czt(c, x, batch, n, ld_x, fs, 0.0, fs * (double)(bins - 1) / (double)n_fft, bins, SPEC_CZT_AUTO,
                        X, ld_X, stream);
    }
    FftPlan p;
    LongPlan lp;
    std::string why, why_long;
    const bool one_pass = fft_plan(batch, n, n_fft, &p, &why, c->fft_cluster);
    if (!one_pass && !long_fft_plan(n, n_fft, &lp, &why_long))
        return fail(c, SPEC_EUNSUPPORTED, why + "; " + why_long);
    if (batch == 0) return SPEC_OK;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!is_device_ptr(x) || !is_device_ptr(X))
        return host_pipeline(c, x, batch, n, ld_x, X, bins, ld_X, st,
                             [&](const float* xd, int64_t ld_xd, float2* Xd, int64_t ld_Xd, int64_t nb) {
                                 return spec_fft(c, xd, nb, n, ld_xd, fs, n_fft, (float*)Xd, ld_Xd, stream);
                             });
    float2* X2 = reinterpret_cast<float2*>(X);
    if (!one_pass) {
        const float2* tw = nullptr;
        float2* work = nullptr;
        int64_t wt = 0;
        if ((s = long_table(c, lp, &tw)) != SPEC_OK) return s;
        if ((s = long_work(c, lp, batch, &work, &wt)) != SPEC_OK) return s;
        cudaError_t e = long_fft_launch(lp, x, batch, (int)n, ld_x, c->block_tw, tw, work, wt, X2, ld_X, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "spec_fft multi-pass launch");
        return SPEC_OK;
    }
    // kernel variants of this shape (compiled two-lane, generic two-lane,
    // one lane, cluster), the fastest chosen by measurement on the first call
    // (autotune.cu); SPEC_LANES pins the lanes and skips the choice
    struct Var {
        FftPlan p;
        int lanes;
    };
    std::vector<Var> vars{{p, c->lanes}};
    std::vector<std::string> names{p.clustered ? "cluster" : p.fixed ? "fixed" : p.dual ? "dual" : "one"};
    if (c->lanes == 0 && p.H > 0) {
        if (p.fixed) {
            FftPlan q = p;
            q.fixed = false;
            vars.push_back({q, 0});
            names.push_back("dual");
            if (fft_fused_available(p.LZ, p.R)) {
                q = p;
                q.fixed = false;
                q.fused = true;
                vars.push_back({q, 0});
                names.push_back("fused");

                if (fft_fused_tma_ok(q, x, (int)n, ld_x)) {
                    vars.push_back({q, 4});
                    names.push_back("fusedp");
                }
            }
            if (fft_fused_available(p.LZ / 2, 2 * p.R, 2)) {
                // residues of LZ/2 points on folded input (k_fft_real_fused, FOLD = 2)
                q = p;
                q.fixed = false;
                q.fused = true;
                q.fold = 2;
                q.LZ = p.LZ / 2;
                q.R = 2 * p.R;
                q.Rc = q.R;
                q.T = q.LZ / 16;
                vars.push_back({q, 0});
                names.push_back("fold");
            }
        }
        if (p.dual || p.fixed) {
            vars.push_back({p, 1});
            names.push_back("one");
        }
        FftPlan q;
        std::string why2;
        if (!p.clustered && fft_plan(batch, n, n_fft, &q, &why2, true) && q.clustered) {
            vars.push_back({q, 0});
            names.push_back("cluster");
        }
    }
    std::vector<const float2*> tabs(vars.size(), nullptr);
    for (size_t i = 0; i < vars.size(); ++i)
        if (vars[i].p.H > 0 && (s = plan_table(c, 0, vars[i].p, &tabs[i])) != SPEC_OK) return s;
    auto run = [&](int i) {
        const Var& v = vars[(size_t)i];
        if (v.lanes == 4)      // the persistent fused kernel (bulk-copy prefetch, bounded waits)
            return fft_fused_tma_launch(v.p, x, batch, ld_x, tabs[(size_t)i], X2, ld_X, c->status,
                                        c->wait_timeout_ns, c->sms, st);
        return fft_launch(v.p, x, batch, (int)n, ld_x, c->block_tw + block_twiddle_offset(v.p.LZ, v.p.emax),
                          tabs[(size_t)i], X2, ld_X, st, v.lanes);
    };
    int pick = 0;
    int pinned = -1;
    for (size_t i = 0; i < names.size() && !c->fft_variant.empty(); ++i)
        if (names[i] == c->fft_variant) pinned = (int)i;
    if (pinned >= 0) {
        pick = pinned;
    } else if (vars.size() > 1) {
        // keyed by shape only: every batch size (and every chunk of a
        // host-buffer call) then runs the same arithmetic
        const std::string key = tune_key("fft", {p.LZ, p.H});
        pick = tune_pick(c, key, names, run, st, &s);
        if (pick < 0) return s == SPEC_OK ? fail(c, SPEC_ECUDA, "spec_fft variant timing") : s;
    }
    cudaError_t e = run(pick);
    if (e != cudaSuccess) return cuda_fail(c, e, "spec_fft launch");
    return SPEC_OK;
}

spec_status spec_czt(spec_ctx* c, const float* x, int64_t batch, int64_t n, int64_t ld_x, double fs,
                     double f1, double f2, int64_t m, int mode, float* X, int64_t ld_X, void* stream) {
    if (!c) return SPEC_EINVAL;
    if (m < 1 || m > (int64_t(1) << 24)) return fail(c, SPEC_EINVAL, "m must be in [1, 2^24]");
    spec_status s = check_common(c, x, batch, n, ld_x, fs, X, m, ld_X);
    if (s != SPEC_OK) return s;
    if (!is_finite(f1) || !is_finite(f2)) return fail(c, SPEC_EINVAL, "f1 and f2 must be finite");
    if (mode < SPEC_CZT_AUTO || mode > SPEC_CZT_GEMM_BF16X1) return fail(c, SPEC_EINVAL, "unknown CZT mode");
    // AUTO is decided on the whole batch (chunks of a host-buffer call then
    // all run the same arithmetic)
    if (mode == SPEC_CZT_AUTO) {
        // measured on a probe batch the first time (n, m, batch size) is
        // seen, then remembered (autotune.cu)
        mode = SPEC_CZT_BLUESTEIN;
        if (batch > 0) {
            DeviceGuard g(c->device);
            spec_status sa = czt_auto_decide(c, batch, n, fs, f1, f2, m, &mode, (cudaStream_t)stream);
            if (sa != SPEC_OK) return sa;
        }
    }
    const bool gemm = mode == SPEC_CZT_GEMM_F16X3 || mode == SPEC_CZT_GEMM_F16X1 || mode == SPEC_CZT_GEMM_BF16X1;
    if (gemm && gemm_z_bytes(n, m) > (size_t(1) << 31))
        return fail(c, SPEC_EUNSUPPORTED, "GEMM chirp-z: Z above 2 GiB (use SPEC_CZT_BLUESTEIN)");
    std::string why, why_long;
    LongPlan lp;
    const bool one_pass = gemm || czt_supported(n, m, &why);
    // N + M - 1 beyond one CTA: with M <= 8192 the trace is cut into segments
    // of P = L' - M + 1 samples that each fit a one-CTA Bluestein of length L'
    // (Section 2.3's sum split over n); otherwise the multi-pass Bluestein.
    const bool segmented = !one_pass && m <= 8192;
    const int seg_L = m <= 2048 ? 8192 : 16384;
    const int64_t seg_P = seg_L - m + 1;
    const int segs = segmented ? (int)((n + seg_P - 1) / seg_P) : 1;
    if (!one_pass && !segmented && !long_czt_plan(n, m, &lp, &why_long))
        return fail(c, SPEC_EUNSUPPORTED, why + "; " + why_long);
    if (batch == 0) return SPEC_OK;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!is_device_ptr(x) || !is_device_ptr(X))
        return host_pipeline(c, x, batch, n, ld_x, X, m, ld_X, st,
                             [&](const float* xd, int64_t ld_xd, float2* Xd, int64_t ld_Xd, int64_t nb) {
                                 return spec_czt(c, xd, nb, n, ld_xd, fs, f1, f2, m, mode, (float*)Xd, ld_Xd,
                                                 stream);
                             });
    if (gemm)
        return czt_gemm(c, x, batch, n, ld_x, fs, f1, f2, m,
                        mode == SPEC_CZT_GEMM_F16X3 ? 3 : mode == SPEC_CZT_GEMM_F16X1 ? 1 : -1, X, ld_X, st);
    float2* X2 = reinterpret_cast<float2*>(X);

    // Bluestein tables for (N, M, f1/fs, step/fs), cached (for a segmented
    // transform: the tables of one segment, N = P)
    const double step = m > 1 ? (f2 - f1) / (double)(m - 1) : 0.0;
    const uint64_t A = cycles_to_fixed(f1 / fs);
    const uint64_t Bh = cycles_to_fixed(0.5 * (step / fs));
    const int64_t n_tab = segmented ? seg_P : n;
    const bool tab_one_pass = one_pass || segmented;
    const int L = one_pass ? czt_length(n, m) : segmented ? seg_L : (1 << lp.logP);
    CztEntry* en = nullptr;
    for (auto& it : c->czt)
        if (it.t.n == n_tab && it.t.m == m && it.t.L == L && it.t.A == A && it.t.Bh == Bh) en = &it;
    if (!en) {
        if (c->czt.size() >= kCztCacheMax) {
            auto lru = std::min_element(c->czt.begin(), c->czt.end(),
                                        [](const CztEntry& a, const CztEntry& b) { return a.last_use < b.last_use; });
            cudaDeviceSynchronize();
            cudaFree(lru->mem);
            cudaEventDestroy(lru->ready);
            c->czt.erase(lru);
        }
        CztEntry ne;
        ne.t.n = (int)n_tab; ne.t.m = (int)m; ne.t.L = L; ne.t.A = A; ne.t.Bh = Bh;
        ne.multipass = !tab_one_pass;
        ne.lp = lp;
        // one allocation: pre[n_tab] | V[L] | post[M] | multi-pass twiddles
        const size_t tw_elems = tab_one_pass ? 0 : (size_t)long_czt_table_entries(lp);
        const size_t off_V = (size_t)n_tab, off_post = off_V + (size_t)L, off_tw = off_post + (size_t)m;
        cudaError_t e = cudaMalloc(&ne.mem, (off_tw + tw_elems) * sizeof(float2));
        if (e != cudaSuccess) return cuda_fail(c, e, "CZT tables");
        ne.t.pre = (float2*)ne.mem;
        ne.t.V = ne.t.pre + off_V;
        ne.t.post = ne.t.pre + off_post;
        if (!tab_one_pass) {
            ne.tw2 = ne.t.pre + off_tw;
            std::vector<float2> host(tw_elems);
            long_fill_tw(lp, host.data());
            e = cudaMemcpy(ne.tw2, host.data(), tw_elems * sizeof(float2), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) { cudaFree(ne.mem); return cuda_fail(c, e, "CZT twiddles"); }
        }
        e = cudaEventCreateWithFlags(&ne.ready, cudaEventDisableTiming);
        if (e != cudaSuccess) { cudaFree(ne.mem); return cuda_fail(c, e, "event"); }
        e = tab_one_pass ? czt_build_tables(ne.t, c->block_tw + block_twiddle_offset(L), st)
                         : long_czt_build_tables(lp, ne.t, c->block_tw, ne.tw2, st);
        if (e == cudaSuccess) e = cudaEventRecord(ne.ready, st);
        if (e != cudaSuccess) {
            cudaFree(ne.mem);
            cudaEventDestroy(ne.ready);
            return cuda_fail(c, e, "CZT table build");
        }
        c->czt.push_back(ne);
        en = &c->czt.back();
    } else {
        cudaError_t e = cudaStreamWaitEvent(st, en->ready, 0);
        if (e != cudaSuccess) return cuda_fail(c, e, "table wait");
    }
    en->last_use = ++c->tick;

    if (segmented) {
        // W: [traces][segs][M] in chunks of at most ~1 GiB
        const int64_t per = (int64_t)segs * m * (int64_t)sizeof(float2);
        const int64_t chunk = std::min<int64_t>(batch, std::max<int64_t>(1, (int64_t(1) << 30) / per));
        if ((s = ensure_stage(c, 3, (size_t)(chunk * per))) != SPEC_OK) return s;
        const uint64_t Bs = cycles_to_fixed(step / fs);
        for (int64_t b0 = 0; b0 < batch; b0 += chunk) {
            const int64_t nb = std::min(chunk, batch - b0);
            cudaError_t e = czt_seg_launch(en->t, x + b0 * ld_x, nb, n, ld_x, (int)seg_P, segs,
                                           c->block_tw + block_twiddle_offset(L), (float2*)c->stage[3], st);
            if (e == cudaSuccess)
                e = czt_combine_launch((const float2*)c->stage[3], segs, (int)m, nb, A, Bs, seg_P, X2 + b0 * ld_X,
                                       ld_X, st);
            if (e != cudaSuccess) return cuda_fail(c, e, "spec_czt segmented launch");
        }
        return SPEC_OK;
    }
    if (en->multipass) {
        float2* work = nullptr;
        int64_t wt = 0;
        if ((s = long_work(c, en->lp, batch, &work, &wt)) != SPEC_OK) return s;
        cudaError_t e = long_czt_launch(en->lp, en->t, en->tw2, x, batch, ld_x, c->block_tw, work, wt, X2,
                                        ld_X, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "spec_czt multi-pass launch");
        return SPEC_OK;
    }
    // one or two traces per thread (packed lanes): pinned by SPEC_LANES, else
    // measured on the first call with this shape (autotune.cu)
    auto run = [&](int i) {
        return i == 1 ? czt_launch2(en->t, x, batch, ld_x, c->block_tw + block_twiddle_offset(L), X2, ld_X, st)
                      : czt_launch(en->t, x, batch, ld_x, c->block_tw + block_twiddle_offset(L), X2, ld_X, st);
    };
    int pick = (czt_dual_ok(L) && c->lanes == 2) ? 1 : 0;
    if (c->lanes == 0 && czt_dual_ok(L) && batch >= 2) {
        const std::string key = tune_key("bluestein", {n, m, L});
        pick = tune_pick(c, key, {"one", "two"}, run, st, &s);
        if (pick < 0) return s == SPEC_OK ? fail(c, SPEC_ECUDA, "spec_czt variant timing") : s;
    }
    cudaError_t e = run(pick);
    if (e != cudaSuccess) return cuda_fail(c, e, "spec_czt launch");
    return SPEC_OK;
}

spec_status spec_czt_spiral(spec_ctx* c, const float* x, int64_t batch, int64_t n, int64_t ld_x, double fs,
                            double f1, double f2, int64_t m, double a0, double w0, float* X, int64_t ld_X,
                            void* stream) {
    if (!c) return SPEC_EINVAL;
    if (m < 1 || m > (int64_t(1) << 24)) return fail(c, SPEC_EINVAL, "m must be in [1, 2^24]");
    spec_status s = check_common(c, x, batch, n, ld_x, fs, X, m, ld_X);
    if (s != SPEC_OK) return s;
    if (!is_finite(f1) || !is_finite(f2)) return fail(c, SPEC_EINVAL, "f1 and f2 must be finite");
    if (!(a0 > 0.0) || !(w0 > 0.0) || !is_finite(a0) || !is_finite(w0))
        return fail(c, SPEC_EINVAL, "a0 and w0 must be positive and finite");
    if (batch > 0 && (!is_device_ptr(x) || !is_device_ptr(X))) {
        // the contour's limits are checked once, before any copy
        if ((s = czt_gemm(c, x, 0, n, ld_x, fs, f1, f2, m, 3, X, ld_X, nullptr, a0, w0)) != SPEC_OK) return s;
        DeviceGuard g(c->device);
        return host_pipeline(c, x, batch, n, ld_x, X, m, ld_X, (cudaStream_t)stream,
                             [&](const float* xd, int64_t ld_xd, float2* Xd, int64_t ld_Xd, int64_t nb) {
                                 return spec_czt_spiral(c, xd, nb, n, ld_xd, fs, f1, f2, m, a0, w0, (float*)Xd,
                                                        ld_Xd, stream);
                             });
    }
    return czt_gemm(c, x, batch, n, ld_x, fs, f1, f2, m, 3, X, ld_X, (cudaStream_t)stream, a0, w0);
}

spec_status spec_zoom(spec_ctx* c, const float* x, int64_t batch, int64_t n, int64_t ld_x, double fs,
                      double f1, double f2, int64_t d, const float* taps, int64_t n_taps, int64_t n_fft,
                      float* X, int64_t ld_X, void* stream) {
    if (!c) return SPEC_EINVAL;
    if (d < 1) return fail(c, SPEC_EINVAL, "d must be >= 1");
    if (n_fft < 1 || n_fft % d != 0 || !is_pow2(n_fft / d) || n_fft / d > (int64_t(1) << 24))
        return fail(c, SPEC_EINVAL, "n_fft must be a multiple of d with n_fft/d a power of two");
    const int64_t K = n_fft / d;
    spec_status s = check_common(c, x, batch, n, ld_x, fs, X, K, ld_X);
    if (s != SPEC_OK) return s;
    if (!taps) return fail(c, SPEC_EINVAL, "taps must not be NULL");
    if (n_taps < 1 || n_taps > 65536) return fail(c, SPEC_EINVAL, "n_taps must be in [1, 65536]");
    if (!is_finite(f1) || !is_finite(f2)) return fail(c, SPEC_EINVAL, "f1 and f2 must be finite");
    if ((n + n_taps - 1 + d - 1) / d > K)
        return fail(c, SPEC_EINVAL, "ceil((n + n_taps - 1)/d) must not exceed n_fft/d");
    ZoomPlan p;
    std::string why;
    if (!zoom_plan(n, d, n_taps, n_fft, fs, f1, f2, &p, &why)) {
        std::string why2;
        if (!zoom_big_plan(batch, n, d, n_taps, n_fft, fs, f1, f2, &p, &why2))
            return fail(c, SPEC_EUNSUPPORTED, why + "; " + why2);
    }
    if (batch == 0) return SPEC_OK;
    DeviceGuard g(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const float* taps_d = taps;
    if (!is_device_ptr(taps)) {
        if ((s = ensure_stage(c, 2, (size_t)n_taps * sizeof(float))) != SPEC_OK) return s;
        cudaError_t e = cudaMemcpyAsync(c->stage[2], taps, n_taps * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy of taps");
        taps_d = (const float*)c->stage[2];
    }
    if (!is_device_ptr(x) || !is_device_ptr(X))
        return host_pipeline(c, x, batch, n, ld_x, X, K, ld_X, st,
                             [&](const float* xd, int64_t ld_xd, float2* Xd, int64_t ld_Xd, int64_t nb) {
                                 return spec_zoom(c, xd, nb, n, ld_xd, fs, f1, f2, d, taps_d, n_taps, n_fft,
                                                  (float*)Xd, ld_Xd, stream);
                             });
    float2* X2 = reinterpret_cast<float2*>(X);
    cudaError_t e;
    if (p.big) {
        const float2* tab = nullptr;
        if ((s = plan_table(c, 1, p.fft, &tab)) != SPEC_OK) return s;
        if ((s = ensure_stage(c, 3, (size_t)batch * p.fft.LZ * sizeof(float2))) != SPEC_OK) return s;
        e = zoom_big_launch(p, x, batch, ld_x, taps_d, (float2*)c->stage[3],
                            c->block_tw + block_twiddle_offset(p.fft.LZ), tab, X2, ld_X, st);
    } else {
        // one or two traces per CTA: pinned by SPEC_LANES, else measured once
        auto run = [&](int i) {
            return zoom_launch(p, x, batch, ld_x, taps_d, c->block_tw + block_twiddle_offset(p.K), X2, ld_X, st,
                               i == 1 ? 2 : 1);
        };
        int pick = c->lanes == 2 ? 1 : 0;
        if (c->lanes == 0 && p.dual && batch >= 2) {
            spec_status ts = SPEC_OK;
            const std::string key = tune_key("zoom", {n, d, n_taps, p.K});
            pick = tune_pick(c, key, {"one", "two"}, run, st, &ts);
            if (pick < 0) return ts == SPEC_OK ? fail(c, SPEC_ECUDA, "spec_zoom variant timing") : ts;
        }
        e = run(pick);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "spec_zoom launch");
    return SPEC_OK;
}

// ---- host helpers ----------------------------------------------------------

int64_t spec_zeros_for_delta(double fs, int64_t n_fft, double delta) {
    if (!(fs > 0.0) || n_fft <= 0 || !(delta >= 0.0) || !(delta * (double)n_fft < fs)) return -1;
    const double N = (double)n_fft;
    const double xr = fs * N / (fs - delta * N) - N;   // Eq. 5
    int64_t x = (int64_t)std::ceil(xr - 1e-9 * std::max(1.0, std::fabs(xr)));
    if (x < 0) x = 0;
    while (fs / N - fs / (N + (double)x) < delta * (1.0 - 1e-12)) ++x;
    return x;
}

int64_t spec_m_for_resolution(double fs, double f1, double f2, int64_t n_fft) {
    if (!(fs > 0.0) || n_fft <= 0) return -1;
    const double v = std::fabs(f2 - f1) / fs * (double)n_fft;   // Eq. 25
    int64_t m = (int64_t)std::ceil(v - 1e-9 * std::max(1.0, v));
    return m < 1 ? 1 : m;
}

spec_status spec_design_lowpass(float* taps, int64_t n_taps, int64_t d) {
    if (!taps || n_taps < 1 || d < 1) return SPEC_EINVAL;
    std::vector<double> h((size_t)n_taps);
    const double pi = 3.14159265358979323846;
    const double mid = 0.5 * (double)(n_taps - 1);
    double sum = 0.0;
    for (int64_t k = 0; k < n_taps; ++k) {
        const double w = n_taps == 1 ? 1.0 : 0.54 - 0.46 * std::cos(2.0 * pi * (double)k / (double)(n_taps - 1));
        const double u = ((double)k - mid) / (double)d;
        const double sinc = u == 0.0 ? 1.0 : std::sin(pi * u) / (pi * u);
        h[(size_t)k] = w * sinc / (double)d;
        sum += h[(size_t)k];
    }
    for (int64_t k = 0; k < n_taps; ++k) taps[k] = (float)(h[(size_t)k] * ((double)d / sum));
    return SPEC_OK;
}

}  // extern "C"
