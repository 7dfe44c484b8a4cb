// autotune.cu -- measured choices for SPEC_CZT_AUTO, remembered per context
// and persisted to a JSON file.
//
// The chirp-z of Section 2.3 has two exact evaluations in this library:
// Bluestein's convolution (Eq. 13-15; segmented or multi-pass for long
// traces) and the direct sum of Eq. 11 as a split-FP16 tensor-core product.
// Which is faster depends on N, M and the batch (tile fill of the product,
// Bluestein length L = nextpow2(N + M - 1)).  SPEC_CZT_AUTO decides per
// (N, M, batch rounded up to a power of two) by running both on a probe batch
// on the device: the product is admitted only if its spectra agree with
// Bluestein's to a relative L2 of 1e-5 per spectrum (both are FP32-level
// accurate, so their difference bounds the product's error at that bar), and
// the faster admitted form wins.  The decision is kept in the context and,
// when SPEC_AUTOTUNE_CACHE names a file, in that file, keyed by a device tag
// (GPU name, multiprocessor count, compute capability, cache format): a file
// written on another device or by another format is ignored and rewritten.
//
// File format (one JSON object; keys and values use only [A-Za-z0-9_.:=| -]):
//   {"format": "spec-autotune-1", "device": "<tag>",
//    "entries": {"czt n=1024 m=512 b=65536": "gemm_f16x3", ...}}
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <fstream>
#include <functional>
#include <vector>
#include <map>
#include <sstream>
#include <string>

#include "ctx.h"
#include "spec.h"
#include "spec_internal.h"

namespace spec {

static const char* kTuneFormat = "spec-autotune-1";

// ---------------------------------------------------------------- file I/O --

namespace {

// a quoted string at s[i] ("..." without escapes); advances i past it
bool read_string(const std::string& s, size_t& i, std::string* out) {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\t' || s[i] == '\r')) ++i;
    if (i >= s.size() || s[i] != '"') return false;
    const size_t j = s.find('"', i + 1);
    if (j == std::string::npos) return false;
    *out = s.substr(i + 1, j - i - 1);
    i = j + 1;
    return true;
}

bool expect(const std::string& s, size_t& i, char c) {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\t' || s[i] == '\r')) ++i;
    if (i >= s.size() || s[i] != c) return false;
    ++i;
    return true;
}

bool peek(const std::string& s, size_t i, char c) {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\t' || s[i] == '\r')) ++i;
    return i < s.size() && s[i] == c;
}

bool safe_text(const std::string& t) {
    for (char ch : t)
        if (!(std::isalnum((unsigned char)ch) || std::strchr("_.:=| -", ch))) return false;
    return !t.empty();
}

}  // namespace

// Parse a cache file.  Returns false (and leaves *entries empty) if the file
// is missing, malformed, of another format or written for another device.
bool tune_file_read(const std::string& path, const std::string& device, std::map<std::string, std::string>* entries) {
    entries->clear();
    std::ifstream f(path);
    if (!f) return false;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    size_t i = 0;
    std::string fmt, dev;
    std::map<std::string, std::string> got;
    if (!expect(s, i, '{')) return false;
    bool have_entries = false;
    for (;;) {
        std::string key;
        if (!read_string(s, i, &key) || !expect(s, i, ':')) return false;
        if (key == "entries") {
            if (!expect(s, i, '{')) return false;
            if (!peek(s, i, '}'))
                for (;;) {
                    std::string k, v;
                    if (!read_string(s, i, &k) || !expect(s, i, ':') || !read_string(s, i, &v)) return false;
                    got[k] = v;
                    if (peek(s, i, ',')) {
                        expect(s, i, ',');
                        continue;
                    }
                    break;
                }
            if (!expect(s, i, '}')) return false;
            have_entries = true;
        } else {
            std::string v;
            if (!read_string(s, i, &v)) return false;
            if (key == "format") fmt = v;
            if (key == "device") dev = v;
        }
        if (peek(s, i, ',')) {
            expect(s, i, ',');
            continue;
        }
        break;
    }
    if (!expect(s, i, '}') || !have_entries || fmt != kTuneFormat || dev != device) return false;
    *entries = got;
    return true;
}

// Write the whole cache (through a temporary file and a rename, so a reader
// never sees half a file).  Entries with characters outside the safe set
// are dropped.
bool tune_file_write(const std::string& path, const std::string& device,
                     const std::map<std::string, std::string>& entries) {
    if (!safe_text(device)) return false;
    const std::string tmp = path + ".tmp";
    {
        std::ofstream f(tmp, std::ios::trunc);
        if (!f) return false;
        f << "{\"format\": \"" << kTuneFormat << "\", \"device\": \"" << device << "\", \"entries\": {";
        bool first = true;
        for (const auto& kv : entries) {
            if (!safe_text(kv.first) || !safe_text(kv.second)) continue;
            f << (first ? "\n  " : ",\n  ") << '"' << kv.first << "\": \"" << kv.second << '"';
            first = false;
        }
        f << "\n}}\n";
        if (!f) return false;
    }
    return std::rename(tmp.c_str(), path.c_str()) == 0;
}

// Store one entry: entries of the same device and format are kept, anything
// else in the file is replaced.
bool tune_file_store(const std::string& path, const std::string& device, const std::string& key,
                     const std::string& value) {
    std::map<std::string, std::string> entries;
    tune_file_read(path, device, &entries);
    entries[key] = value;
    return tune_file_write(path, device, entries);
}

}  // namespace spec

// ------------------------------------------------------ measured decision --

namespace spec {

std::string device_tag(int device) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string name;
    for (const char* q = p.name; *q; ++q)
        name += (std::isalnum((unsigned char)*q) || *q == '-' || *q == '_' || *q == ' ') ? *q : '_';
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s|sm=%d|cc=%d.%d|%s", name.c_str(), p.multiProcessorCount, p.major, p.minor,
                  kTuneFormat);
    return buf;
}

// Deterministic probe traces, uniform in [-1, 1) (splitmix64 of the index).
__global__ void k_probe_fill(float* x, int64_t count, uint64_t seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)i * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[i] = (float)((double)(z >> 11) * 0x1.0p-52 - 1.0);
    }
}

// Per row: ||a - b|| / ||b||; the largest over the rows (as float bits; the
// values are non-negative, so their bit patterns order like the values).
__global__ void k_rel_l2_rows(const float2* a, const float2* b, int64_t cols, unsigned* max_bits) {
    __shared__ double num[256], den[256];
    const float2* ar = a + (int64_t)blockIdx.x * cols;
    const float2* br = b + (int64_t)blockIdx.x * cols;
    double nn = 0.0, dd = 0.0;
    for (int64_t k = threadIdx.x; k < cols; k += 256) {
        const double dx = (double)ar[k].x - br[k].x, dy = (double)ar[k].y - br[k].y;
        nn += dx * dx + dy * dy;
        dd += (double)br[k].x * br[k].x + (double)br[k].y * br[k].y;
    }
    num[threadIdx.x] = nn;
    den[threadIdx.x] = dd;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            num[threadIdx.x] += num[threadIdx.x + w];
            den[threadIdx.x] += den[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float r = den[0] > 0.0 ? (float)std::sqrt(num[0] / den[0]) : (num[0] > 0.0 ? 1e30f : 0.f);
        atomicMax(max_bits, __float_as_uint(r));
    }
}

namespace {

std::string czt_key(int64_t batch, int64_t n, int64_t m) {
    const int64_t b = std::min<int64_t>(next_pow2(std::max<int64_t>(1, batch)), 65536);
    char buf[128];
    std::snprintf(buf, sizeof(buf), "czt n=%lld m=%lld b=%lld", (long long)n, (long long)m, (long long)b);
    return buf;
}

float time_mode(spec_ctx* c, const float* x, int64_t B, int64_t n, double fs, double f1, double f2, int64_t m,
                int mode, float2* X, cudaStream_t st, spec_status* s) {
    cudaEvent_t ea, eb;
    cudaEventCreate(&ea);
    cudaEventCreate(&eb);
    float best = 1e30f;
    for (int r = 0; r < 3 && *s == SPEC_OK; ++r) {
        cudaEventRecord(ea, st);
        *s = spec_czt(c, x, B, n, n, fs, f1, f2, m, mode, reinterpret_cast<float*>(X), m, st);
        cudaEventRecord(eb, st);
        if (*s == SPEC_OK && cudaEventSynchronize(eb) == cudaSuccess) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ea, eb);
            if (r > 0) best = std::min(best, ms);
        }
    }
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    return best;
}

}  // namespace

// The explicit mode SPEC_CZT_AUTO stands for at (batch, n, m): remembered,
// read from the cache file, or measured now (synchronises `st`).
spec_status czt_auto_decide(spec_ctx* c, int64_t batch, int64_t n, double fs, double f1, double f2, int64_t m,
                            int* mode, cudaStream_t st) {
    const std::string key = czt_key(batch, n, m);
    auto it = c->tune.find(key);
    if (it != c->tune.end()) {
        *mode = it->second == "gemm_f16x3" ? SPEC_CZT_GEMM_F16X3 : SPEC_CZT_BLUESTEIN;
        return SPEC_OK;
    }
    *mode = SPEC_CZT_BLUESTEIN;
    // under stream capture nothing can be measured: Bluestein, not remembered
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return SPEC_OK;
    }
    // the product is a candidate when its Z table fits and the batch fills
    // the GPU with output tiles; a model far on Bluestein's side skips it
    bool candidate = gemm_z_bytes(n, m) <= (size_t(1) << 31) &&
                     (batch + 127) / 128 * ((2 * m + 127) / 128) >= std::max(1, c->sms);
    if (candidate) {
        const double L = (double)next_pow2(std::max<int64_t>(16, n + m - 1));
        const double t_gemm = 12.0 * (double)n * (double)m / 1.4e15 + 8.0 * (double)n / 6e12;
        const double t_blue = 0.39e-12 * L * std::log2(L);
        candidate = t_gemm < 4.0 * t_blue;
    }
    std::string value = "bluestein";
    if (candidate) {
        const int64_t per = 4 * n + 16 * m;
        const int64_t B = std::max<int64_t>(1, std::min<int64_t>({batch, 16384, (int64_t(256) << 20) / per}));
        float* xp = nullptr;
        float2 *Xa = nullptr, *Xb = nullptr;
        unsigned* rel = nullptr;
        cudaError_t e = cudaMalloc(&xp, (size_t)B * n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&Xa, (size_t)B * m * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc(&Xb, (size_t)B * m * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc(&rel, sizeof(unsigned));
        spec_status s = SPEC_OK;
        float tb = 1e30f, tg = 1e30f, r = 1e30f;
        if (e == cudaSuccess) {
            k_probe_fill<<<1024, 256, 0, st>>>(xp, B * n, 0x5EC7A11ull);
            e = cudaMemsetAsync(rel, 0, sizeof(unsigned), st);
        }
        if (e == cudaSuccess) {
            tb = time_mode(c, xp, B, n, fs, f1, f2, m, SPEC_CZT_BLUESTEIN, Xa, st, &s);
            if (s == SPEC_OK) tg = time_mode(c, xp, B, n, fs, f1, f2, m, SPEC_CZT_GEMM_F16X3, Xb, st, &s);
            if (s == SPEC_OK) {
                k_rel_l2_rows<<<(unsigned)B, 256, 0, st>>>(Xb, Xa, m, rel);
                unsigned bits = 0;
                e = cudaMemcpyAsync(&bits, rel, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                std::memcpy(&r, &bits, sizeof(float));
            }
        }
        if (xp) cudaFree(xp);
        if (Xa) cudaFree(Xa);
        if (Xb) cudaFree(Xb);
        if (rel) cudaFree(rel);
        if (e != cudaSuccess) return ctx_cuda_fail(c, e, "chirp-z autotune");
        if (s != SPEC_OK) return s;
        if (r <= 1e-5f && tg < tb) {
            value = "gemm_f16x3";
            *mode = SPEC_CZT_GEMM_F16X3;
        }
    }
    c->tune[key] = value;
    if (!c->tune_path.empty()) tune_file_store(c->tune_path, c->tune_device, key, value);
    return SPEC_OK;
}

}  // namespace spec

using namespace spec;

extern "C" spec_status spec_czt_auto_mode(spec_ctx* c, int64_t batch, int64_t n, double fs, double f1, double f2,
                                          int64_t m, int* mode, void* stream) {
    if (!c || !mode || batch < 1 || n < 1 || m < 1 || !(fs > 0.0)) return SPEC_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    const spec_status s = czt_auto_decide(c, batch, n, fs, f1, f2, m, mode, (cudaStream_t)stream);
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return s;
}

extern "C" int spec_tune_cache_store(const char* path, const char* device, const char* key, const char* value) {
    if (!path || !device || !key || !value) return -1;
    return tune_file_store(path, device, key, value) ? 0 : -1;
}

extern "C" int spec_tune_cache_lookup(const char* path, const char* device, const char* key, char* value, int cap) {
    if (!path || !device || !key) return 0;
    std::map<std::string, std::string> entries;
    if (!tune_file_read(path, device, &entries)) return 0;
    auto it = entries.find(key);
    if (it == entries.end()) return 0;
    if (value && cap > 0) {
        std::strncpy(value, it->second.c_str(), (size_t)cap - 1);
        value[cap - 1] = '\0';
    }
    return 1;
}

// ------------------------------------------------- kernel variant choices --

namespace spec {

// The fastest of `names` for `key`: remembered, read from the cache file, or
// measured now by running each candidate three times on the caller's own
// device buffers (the chosen variant then overwrites the output; the first
// run of each is discarded).  Synchronises `st` when it measures.  Returns
// the index into `names`, or -1 with *status set if a candidate fails.
int tune_pick(spec_ctx* c, const std::string& key, const std::vector<std::string>& names,
              const std::function<cudaError_t(int)>& run, cudaStream_t st, spec_status* status) {
    *status = SPEC_OK;
    if (names.size() == 1) return 0;
    auto it = c->tune.find(key);
    if (it != c->tune.end())
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == it->second) return (int)i;
    // nothing can be timed while the stream is being captured into a graph:
    // the first candidate, nothing remembered
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return 0;
    }
    cudaEvent_t ea, eb;
    if (cudaEventCreate(&ea) != cudaSuccess || cudaEventCreate(&eb) != cudaSuccess) {
        cudaGetLastError();
        *status = SPEC_ECUDA;
        return -1;
    }
    int best = -1;
    float best_ms = 1e30f;
    for (size_t i = 0; i < names.size(); ++i) {
        float t = 1e30f;
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(ea, st);
            const cudaError_t e = run((int)i);
            cudaEventRecord(eb, st);
            if (e != cudaSuccess || cudaEventSynchronize(eb) != cudaSuccess) {
                cudaGetLastError();
                t = 1e30f;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ea, eb);
            if (r > 0) t = std::min(t, ms);
        }
        if (t < best_ms) {
            best_ms = t;
            best = (int)i;
        }
    }
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    if (best < 0) {
        *status = SPEC_ECUDA;
        return -1;
    }
    c->tune[key] = names[(size_t)best];
    if (!c->tune_path.empty()) tune_file_store(c->tune_path, c->tune_device, key, names[(size_t)best]);
    return best;
}

// "what v0:v1:..." (the shape a decision belongs to)
std::string tune_key(const char* what, std::initializer_list<long long> v) {
    std::string k = std::string(what) + " ";
    bool first = true;
    for (long long x : v) {
        if (!first) k += ":";
        k += std::to_string(x);
        first = false;
    }
    return k;
}

}  // namespace spec
