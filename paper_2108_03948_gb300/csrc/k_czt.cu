// k_czt.cu -- chirp-z transform on the unit circle by Bluestein's method
// (Section 2.3, Eq. 11-15).
//
// With z_k = e^{j 2 pi (a + b k)}, a = f1/fs, b = step/fs, and the identity
// k n = (k^2 + n^2 - (k - n)^2)/2 (Eq. 12):
//
//   X[k] = post[k] * sum_n (x[n] pre[n]) v[k - n]                (Eq. 13-14)
//   pre[n] = e^{-j 2 pi (a n + (b/2) n^2)},  post[k] = e^{-j 2 pi (b/2) k^2},
//   v[m]  = e^{+j 2 pi (b/2) m^2},  m = -(N-1) .. M-1.
//
// The convolution is circular over a power-of-two L >= N + M - 1 with v
// wrapped (negative m at L + m), evaluated as IFFT(FFT(x pre) * FFT(v))
// (Eq. 15).  FFT(v)/L, pre and post depend only on (N, M, a, b): they are
// built once in float64 from exact fixed-point phases and cached by the
// caller, so each trace costs one FFT and one IFFT, both in shared memory,
// with one HBM read of x and one write of X.
#include "fft_block.cuh"
#include "spec_internal.h"

namespace spec {

__global__ void k_czt_pre_post(float2* pre, int n, float2* post, int m, uint64_t A, uint64_t Bh) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t ii = (uint64_t)i;
    if (i < n) pre[i] = unit_fixed_f64(A * ii + Bh * (ii * ii), true);
    if (i < m) post[i] = unit_fixed_f64(Bh * (ii * ii), true);
}

// V = FFT_L(v)/L for the wrapped chirp kernel v; one CTA.
template <int L>
__global__ void __launch_bounds__(FFTShape<L>::T) k_czt_kernel_spectrum(float2* V, int n, int m, uint64_t Bh,
                                                                       const float2* tw) {
    using FFT = BlockFFT<L, false>;
    constexpr int E = FFT::E, T = FFT::T;
    extern __shared__ float2 smem[];
    const int t = threadIdx.x;
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int idx = t + T * i;
        int64_t mm;
        bool nz = true;
        if (idx < m) mm = idx;
        else if (idx >= L - n + 1) mm = (int64_t)idx - L;
        else { nz = false; mm = 0; }
        const uint64_t m2 = (uint64_t)(mm * mm);
        v[i] = nz ? unit_fixed_f64(Bh * m2, false) : make_float2(0.f, 0.f);
    }
    FFT::run(v, smem, t, tw);
    const float inv = 1.0f / (float)L;
#pragma unroll
    for (int i = 0; i < E; ++i) V[t + T * i] = cscale(v[i], inv);
}

struct BluesteinArgs {
    const float* x;
    int64_t batch;
    int n;
    int64_t ld_x;
    int m;
    const float2* pre;
    const float2* V;
    const float2* post;
    float2* X;
    int64_t ld_X;
    int F;
    const float2* tw;
    const RaggedItem* items;   // ragged batch: per-trace placement, n, m, tables (else null)
    const float2* tables;      // ragged batch: per-trace tables pre | V | post at items[b].tab_off
    int segs;                  // segmented: > 1 segments per trace (batch counts segments)
    int seg_len;               // segmented: samples per segment P
    int64_t n_total;           // segmented: samples per trace N
};

// Up to L = 4096: 256 threads (one or more traces) at four CTAs per SM, i.e.
// 64 registers, which this kernel fits without spills; L = 8192: 512 threads
// at two CTAs per SM (64 registers, no spills; 68 KB of shared memory each).
template <int L>
__global__ void __launch_bounds__(FFTShape<L>::T > 256 ? FFTShape<L>::T : 256,
                                  FFTShape<L>::T > 512 ? 1 : FFTShape<L>::T > 256 ? 2 : 4) k_czt_bluestein(BluesteinArgs a) {
    using Fw = BlockFFT<L, false>;
    using Iv = BlockFFT<L, true>;
    constexpr int E = Fw::E, T = Fw::T;
    extern __shared__ float2 smem[];
    const int f = threadIdx.x / T;
    const int t = threadIdx.x - f * T;
    const int64_t b = (int64_t)blockIdx.x * a.F + f;
    const bool live = b < a.batch;
    float2* s = smem + f * padded_len(L);
    int n = a.n, m = a.m;
    const float2 *pre = a.pre, *V = a.V, *post = a.post;
    int64_t xo = (live ? b : 0) * a.ld_x, Xo = (live ? b : 0) * a.ld_X;
    if (a.items) {
        // a dead slot (b >= batch) borrows trace 0's tables so that the
        // unguarded table reads below stay inside valid memory; its x loads
        // and X stores remain switched off by `live`
        const RaggedItem& it = a.items[live ? b : 0];
        xo = it.x_off;
        Xo = it.out_off;
        n = it.n;
        m = it.m;
        pre = a.tables + it.tab_off;
        V = pre + n;
        post = V + L;
    }
    if (a.segs > 1) {
        // segment sg of trace tr: samples sg P .. sg P + P - 1 (the last may be
        // shorter); its M-point spectrum goes to row b of the workspace
        const int64_t bb = live ? b : 0;
        const int64_t tr = bb / a.segs;
        const int sg = (int)(bb - tr * a.segs);
        xo = tr * a.ld_x + (int64_t)sg * a.seg_len;
        n = (int)min((int64_t)a.seg_len, a.n_total - (int64_t)sg * a.seg_len);
    }
    const float* xr = a.x + xo;

    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int nn = t + T * i;
        v[i] = (live && nn < n) ? cscale(__ldg(&pre[nn]), __ldg(xr + nn)) : make_float2(0.f, 0.f);
    }
    Fw::run(v, s, t, a.tw);
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = cmul(v[i], __ldg(&V[t + T * i]));
    int ti = t;                        // opaque copy: see k_czt_bluestein2
    asm volatile("" : "+r"(ti));
    float2* Xr = a.X + Xo;
    // A uniform batch (one M for every trace of the CTA) with M <= L/4 keeps
    // only outputs t + T i with i < E/4: stored from a separate copy of the
    // inverse FFT, whose unused last-pass outputs the compiler then drops.
    // The choice depends on kernel arguments only, so every thread of the
    // CTA takes the same branch (the FFT holds CTA barriers).
    // (For L >= 4096 only: the second copy makes the smaller sizes spill
    // at 64 registers.)
    if constexpr (L >= 4096) {
        if (!a.items && a.m <= L / 4) {
            Iv::run(v, s, ti, a.tw);
#pragma unroll
            for (int i = 0; i < E / 4; ++i) {
                const int k = t + T * i;
                if (live && k < m) Xr[k] = cmul(v[i], __ldg(&post[k]));
            }
            return;
        }
    }
    Iv::run(v, s, ti, a.tw);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int k = t + T * i;
        if (live && k < m) Xr[k] = cmul(v[i], __ldg(&post[k]));
    }
}

// Two-lane variant: traces 2p and 2p+1 ride in the two packed lanes of a C2,
// so every table value (pre, V, post, twiddles) is loaded once per pair and
// each FFT instruction serves both traces.
template <int L>
__global__ void __launch_bounds__(FFTShape<L>::T > 256 ? FFTShape<L>::T : 256, FFTShape<L>::T > 256 ? 1 : 2)
    k_czt_bluestein2(BluesteinArgs a) {
    using Fw = BlockFFT<L, false, C2>;
    using Iv = BlockFFT<L, true, C2>;
    constexpr int E = Fw::E, T = Fw::T;
    extern __shared__ float4 smem4[];
    const int f = threadIdx.x / T;
    const int t = threadIdx.x - f * T;
    const int64_t b0 = ((int64_t)blockIdx.x * a.F + f) * 2, b1 = b0 + 1;
    const bool live0 = b0 < a.batch, live1 = b1 < a.batch;
    float4* s = smem4 + f * padded_len(L);
    const float* x0 = a.x + (live0 ? b0 : 0) * a.ld_x;
    const float* x1 = a.x + (live1 ? b1 : 0) * a.ld_x;

    C2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int nn = t + T * i;
        if (i % 4 == 0) asm volatile("" ::: "memory");
        if (nn < a.n) {
            const float2 p = __ldg(&a.pre[nn]);
            const float2 xx = make_float2(live0 ? __ldg(x0 + nn) : 0.f, live1 ? __ldg(x1 + nn) : 0.f);
            v[i] = C2{mul2(make_float2(p.x, p.x), xx), mul2(make_float2(p.y, p.y), xx)};
        } else {
            v[i] = C2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        }
    }
    Fw::run(v, s, t, a.tw);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        if (i % 4 == 0) asm volatile("" ::: "memory");   // bound the hoisted float4 loads
        v[i] = mul_tw<false>(v[i], __ldg(&a.V[t + T * i]));
    }
    // an opaque copy of t: the inverse FFT recomputes its shared-memory
    // addresses instead of keeping the forward FFT's alive (register pressure)
    int ti = t;
    asm volatile("" : "+r"(ti));
    Iv::run(v, s, ti, a.tw);
    float2* X0 = a.X + (live0 ? b0 : 0) * a.ld_X;
    float2* X1 = a.X + (live1 ? b1 : 0) * a.ld_X;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int k = t + T * i;
        if (i % 4 == 0) asm volatile("" ::: "memory");
        if (k < a.m) {
            const C2 r = mul_tw<false>(v[i], __ldg(&a.post[k]));
            if (live0) X0[k] = lane_a(r);
            if (live1) X1[k] = lane_b(r);
        }
    }
}

using BsKernel = void (*)(BluesteinArgs);
using VKernel = void (*)(float2*, int, int, uint64_t, const float2*);

template <int L> static void pick(int want, BsKernel* bk, VKernel* vk) {
    if (want == L) { *bk = k_czt_bluestein<L>; *vk = k_czt_kernel_spectrum<L>; }
}

static bool kernels_for(int L, BsKernel* bk, VKernel* vk) {
    *bk = nullptr; *vk = nullptr;
    pick<16>(L, bk, vk); pick<32>(L, bk, vk); pick<64>(L, bk, vk); pick<128>(L, bk, vk);
    pick<256>(L, bk, vk); pick<512>(L, bk, vk); pick<1024>(L, bk, vk); pick<2048>(L, bk, vk);
    pick<4096>(L, bk, vk); pick<8192>(L, bk, vk); pick<16384>(L, bk, vk);
    return *bk != nullptr;
}

int czt_length(int64_t n, int64_t m) { return (int)std::max<int64_t>(16, next_pow2(n + m - 1)); }

bool czt_supported(int64_t n, int64_t m, std::string* why) {
    if (n + m - 1 > 16384) {
        *why = "CZT: N + M - 1 above 16384 needs the multi-pass Bluestein path";
        return false;
    }
    return true;
}

cudaError_t czt_pre_post_launch(const CztTables& t, cudaStream_t st) {
    const int cnt = std::max(t.n, t.m);
    k_czt_pre_post<<<(cnt + 255) / 256, 256, 0, st>>>(t.pre, t.n, t.post, t.m, t.A, t.Bh);
    return cudaGetLastError();
}

cudaError_t czt_build_tables(const CztTables& t, const float2* tw, cudaStream_t st) {
    BsKernel bk;
    VKernel vk;
    if (!kernels_for(t.L, &bk, &vk)) return cudaErrorInvalidValue;
    const int cnt = std::max(t.n, t.m);
    k_czt_pre_post<<<(cnt + 255) / 256, 256, 0, st>>>(t.pre, t.n, t.post, t.m, t.A, t.Bh);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)padded_len(t.L) * sizeof(float2);
    e = cudaFuncSetAttribute(vk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int T = t.L / 16;
    vk<<<1, T, smem, st>>>(t.V, t.n, t.m, t.Bh, tw);
    return cudaGetLastError();
}

cudaError_t czt_launch(const CztTables& t, const float* x, int64_t batch, int64_t ld_x,
                       const float2* tw, float2* X, int64_t ld_X, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    BsKernel bk;
    VKernel vk;
    if (!kernels_for(t.L, &bk, &vk)) return cudaErrorInvalidValue;
    const int T = t.L / 16;
    int F = std::max(1, 256 / T);
    F = (int)std::min<int64_t>(F, batch);
    const size_t smem = (size_t)F * padded_len(t.L) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(bk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    BluesteinArgs a = {};
    a.x = x; a.batch = batch; a.n = t.n; a.ld_x = ld_x; a.m = t.m;
    a.pre = t.pre; a.V = t.V; a.post = t.post; a.X = X; a.ld_X = ld_X; a.F = F; a.tw = tw;
    const int64_t grid = (batch + F - 1) / F;
    bk<<<(unsigned)grid, F * T, smem, st>>>(a);
    return cudaGetLastError();
}

// Segmented chirp-z for N >> M: the trace is cut into S segments of P samples
// and X[k] = sum_s z_k^{-s P} X_s[k] (Eq. 11 split over n = s P + n'), where
// X_s is the chirp-z of segment s by the Bluestein kernel above (tables for
// N = P, shared by every segment).  W holds X_s for every (trace, segment).
cudaError_t czt_seg_launch(const CztTables& t, const float* x, int64_t batch, int64_t n_total, int64_t ld_x,
                           int seg_len, int segs, const float2* tw, float2* W, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    BsKernel bk;
    VKernel vk;
    if (!kernels_for(t.L, &bk, &vk)) return cudaErrorInvalidValue;
    const int T = t.L / 16;
    const int64_t virt = batch * segs;
    int F = std::max(1, 256 / T);
    F = (int)std::min<int64_t>(F, virt);
    const size_t smem = (size_t)F * padded_len(t.L) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(bk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    BluesteinArgs a = {};
    a.x = x; a.batch = virt; a.n = t.n; a.ld_x = ld_x; a.m = t.m;
    a.pre = t.pre; a.V = t.V; a.post = t.post; a.X = W; a.ld_X = t.m; a.F = F; a.tw = tw;
    a.segs = segs; a.seg_len = seg_len; a.n_total = n_total;
    bk<<<(unsigned)((virt + F - 1) / F), F * T, smem, st>>>(a);
    return cudaGetLastError();
}

// X[b][k] = sum_s W[b s][k] e^{-j 2 pi (a + b_step k) s P}: the phase in
// cycles is A s P + B k s P modulo one, exact in 64-bit fixed point
// (A = frac(f1/fs), B = frac(step/fs)).
__global__ void k_czt_combine(const float2* __restrict__ W, int segs, int m, int64_t batch, uint64_t A, uint64_t B,
                              int64_t seg_len, float2* X, int64_t ld_X) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= batch * m) return;
    const int64_t b = idx / m;
    const int k = (int)(idx - b * m);
    const float2* w = W + b * segs * (int64_t)m + k;
    float2 acc = make_float2(0.f, 0.f);
    for (int sg = 0; sg < segs; ++sg) {
        const uint64_t sp = (uint64_t)sg * (uint64_t)seg_len;
        const float2 rot = unit_fixed(A * sp + B * ((uint64_t)k * sp), true);
        acc = cadd(acc, cmul(__ldg(w + (int64_t)sg * m), rot));
    }
    X[b * ld_X + k] = acc;
}

cudaError_t czt_combine_launch(const float2* W, int segs, int m, int64_t batch, uint64_t A, uint64_t B,
                               int64_t seg_len, float2* X, int64_t ld_X, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    const int64_t total = batch * m;
    k_czt_combine<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(W, segs, m, batch, A, B, seg_len, X, ld_X);
    return cudaGetLastError();
}

template <int L> static void pick2(int want, BsKernel* bk) {
    if (want == L) *bk = k_czt_bluestein2<L>;
}

static bool kernel2_for(int L, BsKernel* bk) {
    *bk = nullptr;
    pick2<16>(L, bk); pick2<32>(L, bk); pick2<64>(L, bk); pick2<128>(L, bk); pick2<256>(L, bk);
    pick2<512>(L, bk); pick2<1024>(L, bk); pick2<2048>(L, bk); pick2<4096>(L, bk); pick2<8192>(L, bk);
    return *bk != nullptr;
}

bool czt_dual_ok(int L) { return L >= 16 && L <= 8192; }

cudaError_t czt_launch2(const CztTables& t, const float* x, int64_t batch, int64_t ld_x,
                        const float2* tw, float2* X, int64_t ld_X, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    BsKernel bk;
    if (!kernel2_for(t.L, &bk)) return cudaErrorInvalidValue;
    const int T = t.L / 16;
    const int64_t pairs = (batch + 1) / 2;
    int F = std::max(1, 256 / T);
    F = (int)std::min<int64_t>(F, pairs);
    const size_t smem = (size_t)F * padded_len(t.L) * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(bk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    BluesteinArgs a = {};
    a.x = x; a.batch = batch; a.n = t.n; a.ld_x = ld_x; a.m = t.m;
    a.pre = t.pre; a.V = t.V; a.post = t.post; a.X = X; a.ld_X = ld_X; a.F = F;
    a.tw = tw;
    const int64_t grid = (pairs + F - 1) / F;
    bk<<<(unsigned)grid, F * T, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Ragged batches: every trace has its own (N, M, band), so its tables
// pre | V | post live at items[b].tab_off of one buffer; built once per plan.
__global__ void k_czt_pre_post_ragged(const RaggedItem* items, float2* tables, int L) {
    const RaggedItem it = items[blockIdx.x];
    float2* pre = tables + it.tab_off;
    float2* post = pre + it.n + L;
    const int cnt = max(it.n, it.m);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint64_t ii = (uint64_t)i;
        if (i < it.n) pre[i] = unit_fixed_f64(it.A * ii + it.B * (ii * ii), true);
        if (i < it.m) post[i] = unit_fixed_f64(it.B * (ii * ii), true);
    }
}

template <int L>
__global__ void __launch_bounds__(FFTShape<L>::T) k_czt_kernel_spectrum_ragged(const RaggedItem* items, float2* tables,
                                                                              const float2* tw) {
    using FFT = BlockFFT<L, false>;
    constexpr int E = FFT::E, T = FFT::T;
    extern __shared__ float2 smem[];
    const RaggedItem it = items[blockIdx.x];
    const int t = threadIdx.x;
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int idx = t + T * i;
        int64_t mm;
        bool nz = true;
        if (idx < it.m) mm = idx;
        else if (idx >= L - it.n + 1) mm = (int64_t)idx - L;
        else { nz = false; mm = 0; }
        v[i] = nz ? unit_fixed_f64(it.B * (uint64_t)(mm * mm), false) : make_float2(0.f, 0.f);
    }
    FFT::run(v, smem, t, tw);
    float2* V = tables + it.tab_off + it.n;
    const float inv = 1.0f / (float)L;
#pragma unroll
    for (int i = 0; i < E; ++i) V[t + T * i] = cscale(v[i], inv);
}

using VRagged = void (*)(const RaggedItem*, float2*, const float2*);

template <int L> static void pickr(int want, BsKernel* bk, VRagged* vk) {
    if (want == L) { *bk = k_czt_bluestein<L>; *vk = k_czt_kernel_spectrum_ragged<L>; }
}

static bool ragged_kernels_for(int L, BsKernel* bk, VRagged* vk) {
    *bk = nullptr; *vk = nullptr;
    pickr<16>(L, bk, vk); pickr<32>(L, bk, vk); pickr<64>(L, bk, vk); pickr<128>(L, bk, vk);
    pickr<256>(L, bk, vk); pickr<512>(L, bk, vk); pickr<1024>(L, bk, vk); pickr<2048>(L, bk, vk);
    pickr<4096>(L, bk, vk); pickr<8192>(L, bk, vk); pickr<16384>(L, bk, vk);
    return *bk != nullptr;
}

cudaError_t czt_ragged_tables(int L, const RaggedItem* items, int64_t count, float2* tables, const float2* tw,
                              cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    BsKernel bk;
    VRagged vk;
    if (!ragged_kernels_for(L, &bk, &vk)) return cudaErrorInvalidValue;
    k_czt_pre_post_ragged<<<(unsigned)count, 256, 0, st>>>(items, tables, L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)padded_len(L) * sizeof(float2);
    e = cudaFuncSetAttribute(vk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    vk<<<(unsigned)count, L / 16, smem, st>>>(items, tables, tw);
    return cudaGetLastError();
}

cudaError_t czt_ragged_launch(int L, const RaggedItem* items, int64_t count, const float* x_pool,
                              const float2* tables, const float2* tw, float2* X_pool, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    BsKernel bk;
    VRagged vk;
    if (!ragged_kernels_for(L, &bk, &vk)) return cudaErrorInvalidValue;
    const int T = L / 16;
    int F = std::max(1, 256 / T);
    F = (int)std::min<int64_t>(F, count);
    const size_t smem = (size_t)F * padded_len(L) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(bk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    BluesteinArgs a = {};
    a.x = x_pool; a.batch = count; a.X = X_pool; a.F = F; a.tw = tw;
    a.items = items; a.tables = tables;
    bk<<<(unsigned)((count + F - 1) / F), F * T, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Ragged batches as one persistent launch (work queue).  Every trace has its
// own (N, M, band); its Bluestein length L = nextpow2(N + M - 1) <= 16384.
// A unit of work is 16384/L traces of one L, so every unit holds 16384 FFT
// points and runs on the same 1024-thread CTA (16 elements per thread, one
// trace per group of L/16 threads).  The units are sorted by length (largest
// first) on the host and popped from an atomic counter by persistent CTAs,
// one per SM.  The chirps of Eq. 13-15 are evaluated in the kernel from the
// exact 64-bit fixed-point phases (pre[n] = e^{-j2pi(A n + B n^2)}, post[k] =
// e^{-j2pi B k^2}); only FFT(v)/L, which depends on (N, M, B) alone, comes
// from a table, one per distinct (N, M, B) of the batch.
struct CztQueueArgs {
    const RaggedItem* items;   // tab_off: offset of the trace's FFT(v)/L in vpool
    const CztUnit* units;
    int nunits;
    unsigned* counter;         // zeroed before the launch
    const float* x;
    const float2* vpool;
    float2* X;
    const float2* tw;          // BlockFFT twiddles of every size (radix-16 layout)
    const float2* tw32;        // the same for radix-32 passes
};

constexpr int kCztUnitPoints = 8192;
constexpr int kCztQueueThreads = kCztUnitPoints / 16;
// the longest length runs one trace per unit with 32 elements per thread
template <int L> struct CztQueueShape { static constexpr int EMAX = L > kCztUnitPoints ? 32 : 16; };

// The trace of this thread's group, looked up again from opaque copies of the
// unit index and thread index, so that nothing but the FFT data stays live
// across the transforms (64 registers at 1024 threads).
template <int L>
__device__ __forceinline__ const RaggedItem* czt_queue_item(const CztQueueArgs& a, int ui, bool* live) {
    constexpr int T = FFTShape<L, CztQueueShape<L>::EMAX>::T;
    unsigned tid;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
    asm volatile("" : "+r"(ui));
    const int f = (int)tid / T;
    const CztUnit u = a.units[ui];
    *live = f < u.count;
    return a.items + u.first + (*live ? f : 0);
}

template <int L>
__device__ __forceinline__ void czt_queue_unit(const CztQueueArgs& a, int ui, float2* smem) {
    constexpr int EMAX = CztQueueShape<L>::EMAX;
    using Fw = BlockFFT<L, false, float2, EMAX>;
    using Iv = BlockFFT<L, true, float2, EMAX>;
    constexpr int E = Fw::E, T = Fw::T;
    constexpr int SL = L + L / EMAX;                      // padded slots of one trace
    const int f = threadIdx.x / T;
    const int t = threadIdx.x - f * T;
    const float2* tw = (EMAX == 32 ? a.tw32 : a.tw) + fft_twiddle_offset(L, EMAX);
    float2* s = smem + f * SL;
    // The chirps are evaluated while no FFT data is live in registers: the
    // chirped input goes through this thread's own slots of the shared
    // FFT area (read back before the FFT's first barrier), and the inverse
    // FFT's outputs come back through the same slots.
    {
        bool live;
        const RaggedItem* it = czt_queue_item<L>(a, ui, &live);
        const float* xr = a.x + it->x_off;
        const int n = it->n;
        const uint64_t A = it->A, B = it->B;
        for (int i = 0; i < E; ++i) {
            const int nn = t + T * i;
            const uint64_t q = (uint64_t)nn;
            s[pidx_p<EMAX>(nn)] = (live && nn < n) ? cscale(unit_fast(A * q + B * (q * q), true), __ldg(xr + nn))
                                                   : make_float2(0.f, 0.f);
        }
    }
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = s[pidx_p<EMAX>(t + T * i)];
    Fw::run(v, s, t, tw);
    {
        bool live;
        const float2* V = a.vpool + czt_queue_item<L>(a, ui, &live)->tab_off;
        unsigned tt;
        asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tt));
        V += (int)(tt % T);
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = cmul(v[i], __ldg(V + T * i));
    }
    int t2 = t;
    asm volatile("" : "+r"(t2));
    Iv::run(v, s, t2, tw);
    unsigned tid;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
    const int t3 = (int)(tid % T);
    float2* s3 = smem + (int)(tid / T) * SL;
#pragma unroll
    for (int i = 0; i < E; ++i) s3[pidx_p<EMAX>(t3 + T * i)] = v[i];
    bool live;
    const RaggedItem* it = czt_queue_item<L>(a, ui, &live);
    if (!live) return;
    float2* Xr = a.X + it->out_off;
    const int m = it->m;
    const uint64_t B = it->B;
    for (int i = 0; i < E; ++i) {
        const int k = t3 + T * i;
        const uint64_t q = (uint64_t)k;
        if (k < m) Xr[k] = cmul(s3[pidx_p<EMAX>(k)], unit_fast(B * (q * q), true));
    }
}

__global__ void __launch_bounds__(kCztQueueThreads, 1) k_czt_queue(CztQueueArgs a) {
    extern __shared__ float2 smem[];
    __shared__ int s_unit;
    for (;;) {
        __syncthreads();                              // the previous unit is done with s_unit and smem
        if (threadIdx.x == 0) s_unit = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int ui = s_unit;
        if (ui >= a.nunits) return;
        switch (a.units[ui].L) {
            case 16: czt_queue_unit<16>(a, ui, smem); break;
            case 32: czt_queue_unit<32>(a, ui, smem); break;
            case 64: czt_queue_unit<64>(a, ui, smem); break;
            case 128: czt_queue_unit<128>(a, ui, smem); break;
            case 256: czt_queue_unit<256>(a, ui, smem); break;
            case 512: czt_queue_unit<512>(a, ui, smem); break;
            case 1024: czt_queue_unit<1024>(a, ui, smem); break;
            case 2048: czt_queue_unit<2048>(a, ui, smem); break;
            case 4096: czt_queue_unit<4096>(a, ui, smem); break;
            case 8192: czt_queue_unit<8192>(a, ui, smem); break;
            default: czt_queue_unit<16384>(a, ui, smem); break;
        }
    }
}

// FFT(v)/L of one distinct (N, M, B) per CTA, written at items[b].tab_off of
// vpool: v[m] = e^{+j2pi B m^2} for m in [-(N-1), M-1], wrapped circularly.
template <int L>
__global__ void __launch_bounds__(FFTShape<L>::T) k_czt_vpool(const RaggedItem* keys, float2* vpool, const float2* tw) {
    using FFT = BlockFFT<L, false>;
    constexpr int E = FFT::E, T = FFT::T;
    extern __shared__ float2 smem[];
    const RaggedItem it = keys[blockIdx.x];
    const int t = threadIdx.x;
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int idx = t + T * i;
        int64_t mm = 0;
        bool nz = true;
        if (idx < it.m) mm = idx;
        else if (idx >= L - it.n + 1) mm = (int64_t)idx - L;
        else nz = false;
        v[i] = nz ? unit_fixed_f64(it.B * (uint64_t)(mm * mm), false) : make_float2(0.f, 0.f);
    }
    FFT::run(v, smem, t, tw);
    const float inv = 1.0f / (float)L;
    float2* V = vpool + it.tab_off;
#pragma unroll
    for (int i = 0; i < E; ++i) V[t + T * i] = cscale(v[i], inv);
}

using VPoolKernel = void (*)(const RaggedItem*, float2*, const float2*);

static VPoolKernel vpool_kernel_for(int L) {
    switch (L) {
        case 16: return k_czt_vpool<16>;
        case 32: return k_czt_vpool<32>;
        case 64: return k_czt_vpool<64>;
        case 128: return k_czt_vpool<128>;
        case 256: return k_czt_vpool<256>;
        case 512: return k_czt_vpool<512>;
        case 1024: return k_czt_vpool<1024>;
        case 2048: return k_czt_vpool<2048>;
        case 4096: return k_czt_vpool<4096>;
        case 8192: return k_czt_vpool<8192>;
        case 16384: return k_czt_vpool<16384>;
        default: return nullptr;
    }
}

cudaError_t czt_vpool_build(int L, const RaggedItem* keys, int64_t count, float2* vpool, const float2* tw_base,
                            cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    VPoolKernel k = vpool_kernel_for(L);
    if (!k) return cudaErrorInvalidValue;
    const size_t smem = (size_t)padded_len(L) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)count, std::max(1, L / 16), smem, st>>>(keys, vpool, tw_base + (L <= 16 ? 0 : fft_twiddle_offset(L)));
    return cudaGetLastError();
}

size_t czt_queue_smem() { return (size_t)(2 * kCztUnitPoints + 2 * kCztUnitPoints / 32) * sizeof(float2); }
int czt_queue_unit_traces(int L) { return L >= kCztUnitPoints ? 1 : kCztUnitPoints / L; }

// One persistent launch over the unit list; `counter` must be zero (the
// caller's graph zeroes it before the launch).
cudaError_t czt_queue_launch(const RaggedItem* items, const CztUnit* units, int nunits, unsigned* counter,
                             const float* x_pool, const float2* vpool, const float2* tw_base, const float2* tw32_base,
                             float2* X_pool, int ctas, cudaStream_t st) {
    if (nunits == 0) return cudaSuccess;
    const size_t smem = czt_queue_smem();
    cudaError_t e = cudaFuncSetAttribute(k_czt_queue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    CztQueueArgs a = {};
    a.items = items; a.units = units; a.nunits = nunits; a.counter = counter;
    a.x = x_pool; a.vpool = vpool; a.X = X_pool; a.tw = tw_base; a.tw32 = tw32_base;
    k_czt_queue<<<(unsigned)std::max(1, std::min(ctas, nunits)), kCztQueueThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace spec
