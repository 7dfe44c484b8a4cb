// czt_static.cu -- spec_czt_static: the chirp-z transform (Bluestein) for
// callers that cannot allocate device memory.
//
// Who needs it: code whose device memory belongs to someone else -- a
// framework's caching allocator that has reserved the pool, a real-time loop
// that must not call cudaMalloc (it can synchronise the device and its
// latency is unbounded), a plug-in that is handed buffers but no allocator.
// spec_czt needs a context, and a context allocates its tables with
// cudaMalloc; this entry point needs neither.
//
// Its working memory is the file-scope array g_czt_scratch below, a fixed
// kStaticScratch complex elements (about 320 KiB) that every GPU loading the
// library keeps until the process exits.  In host code the array's name is
// only a host-side stand-in, so the device address is fetched once per
// device with cudaGetSymbolAddress (with that device current) and passed to
// the kernels.  The first call on a device does that set-up, fills the FFT
// twiddle part of the array and synchronises the caller's stream; make that
// first call before any stream capture.
//
// The cached address and the twiddles belong to the device's current CUDA
// context: after cudaDeviceReset the array is reloaded (zeroed, possibly at
// another address) while the cache still says "set up", so this entry point
// must not be used across a cudaDeviceReset in the same process.
//
// Every call shares the array and leaves its tables there.  Nothing in it
// has to start at zero: each call rewrites the chirp tables and the kernel
// spectrum it reads.  Two calls that run at the same time on the GPU (say on
// two streams) overwrite each other's tables: order them on one stream.
#include <mutex>

#include "fft_block.cuh"
#include "spec.h"
#include "spec_internal.h"

namespace spec {
namespace {

constexpr int kStaticMaxL = 8192;                                   // N + M - 1 <= 8192
constexpr int kStaticTw = fft_twiddle_offset(kStaticMaxL) + fft_twiddle_entries(kStaticMaxL);
constexpr int kStaticScratch = kStaticTw + 3 * kStaticMaxL;         // twiddles | pre | V | post
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_czt_scratch[kStaticScratch];

std::mutex g_mu;
float2* g_scratch[kMaxDevices] = {};   // device address of g_czt_scratch, per device

// Twiddles of every BlockFFT size 32 .. kStaticMaxL (the FFTShape layout),
// float64 from the exact rational angle; one thread per entry.
__global__ void k_static_twiddles(float2* tw, int total) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int LF = 32;
    while (LF < kStaticMaxL && e >= fft_twiddle_offset(LF << 1)) LF <<= 1;
    const int local = e - fft_twiddle_offset(LF);       // NS - 16 + (r-1) NS + k
    int lg = 0;
    while ((1 << lg) < LF) ++lg;
    const int np16 = lg / 4, rem = 1 << (lg % 4);
    int ns = 16;
    for (int p = 1; p < np16 + (rem > 1 ? 1 : 0); ++p) {
        const int R = p < np16 ? 16 : rem;
        const int off = ns - 16;
        if (local < off + (R - 1) * ns) {
            const int r = (local - off) / ns + 1, k = (local - off) % ns;
            const long long S = (long long)ns * R;
            double s, c;
            sincospi(2.0 * (double)(((long long)r * k) % S) / (double)S, &s, &c);
            tw[e] = make_float2((float)c, (float)-s);
            return;
        }
        ns *= R;
    }
}

float2* scratch_for_current_device(cudaStream_t st, spec_status* status) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        *status = SPEC_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch[dev]) return g_scratch[dev];
    float2* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_czt_scratch);
    if (e == cudaSuccess) {
        k_static_twiddles<<<(kStaticTw + 255) / 256, 256, 0, st>>>(ptr, kStaticTw);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *status = SPEC_ECUDA;
        return nullptr;
    }
    g_scratch[dev] = ptr;
    return ptr;
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace spec

using namespace spec;

extern "C" spec_status spec_czt_static(const float* x, int64_t batch, int64_t n, int64_t ld_x, double fs,
                                       double f1, double f2, int64_t m, float* X, int64_t ld_X,
                                       void* stream) {
    if (!x || !X || batch < 0 || n < 1 || m < 1 || ld_x < n || ld_X < m) return SPEC_EINVAL;
    if (!(fs > 0.0) || !std::isfinite(fs) || !std::isfinite(f1) || !std::isfinite(f2)) return SPEC_EINVAL;
    // n and m are bounded first, so that n + m - 1 cannot overflow
    if (n > kStaticMaxL || m > kStaticMaxL || n + m - 1 > kStaticMaxL) return SPEC_EUNSUPPORTED;
    if (batch == 0) return SPEC_OK;
    const uintptr_t px = (uintptr_t)x, pX = (uintptr_t)X;
    const uintptr_t bx = (uintptr_t)(((batch - 1) * ld_x + n) * sizeof(float));
    const uintptr_t bX = (uintptr_t)(((batch - 1) * ld_X + m) * sizeof(float2));
    if (px < pX + bX && pX < px + bx) return SPEC_EINVAL;
    // host buffers would need staging memory: device pointers only
    if (!on_device(x) || !on_device(X)) return SPEC_EINVAL;

    cudaStream_t st = (cudaStream_t)stream;
    spec_status status = SPEC_OK;
    float2* base = scratch_for_current_device(st, &status);
    if (!base) return status;

    CztTables t;
    t.n = (int)n;
    t.m = (int)m;
    t.L = czt_length(n, m);
    const double step = m > 1 ? (f2 - f1) / (double)(m - 1) : 0.0;
    t.A = cycles_to_fixed(f1 / fs);
    t.Bh = cycles_to_fixed(0.5 * (step / fs));
    t.pre = base + kStaticTw;
    t.V = t.pre + kStaticMaxL;
    t.post = t.V + kStaticMaxL;
    const float2* tw = base + (t.L <= 16 ? 0 : fft_twiddle_offset(t.L));
    cudaError_t e = czt_build_tables(t, tw, st);
    if (e == cudaSuccess) e = czt_launch(t, x, batch, ld_x, tw, reinterpret_cast<float2*>(X), ld_X, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SPEC_ECUDA;
    }
    return SPEC_OK;
}
