// k_zoom.cu -- Zoom FFT (Section 2.2, Eq. 6-10): mix the band centre f_N to
// DC, low-pass FIR, keep every D-th sample, K-point FFT, ascending order.
//
// One CTA per trace, one HBM read of x and one write of the K bins.  The
// mix is folded into the taps, which is the same sum regrouped:
//
//   u[m] = sum_k h[k] x[mD-k] e^{-j w (mD-k)}
//        = e^{-j w mD} sum_k (h[k] e^{+j w k}) x[mD-k],   w = 2 pi f_N/fs,
//
// so the FIR runs on the real samples with complex taps g[k] and one
// rotation per kept output.  Only the L_out = ceil((N + L_h - 1)/D) outputs
// that are kept are computed.  The trace sits in shared memory split by
// phase (x[iD + p] at row p, column i) so that the lanes of a warp, which
// compute consecutive outputs m, read consecutive words for every tap; each
// thread computes four outputs per pass over the taps, so a tap is read once
// per four multiply-adds.  Both phases (w k and w mD) are exact 64-bit
// fixed-point products.
#include "fft_block.cuh"
#include "spec_internal.h"

namespace spec {

struct ZoomArgs {
    const float* x;
    int64_t batch;
    int n;
    int64_t ld_x;
    const float* taps;
    int n_taps, d, logd, lout, rs;
    uint64_t Cn;
    const float2* tw;
    float2* X;
    int64_t ld_X;
    const RaggedItem* items;   // ragged batch: per-trace placement and parameters (else null)
};

constexpr int kZoomGroup = 4;   // outputs per thread per pass over the taps (at most)

// FIR + decimate of one trace: thread t computes the G outputs
// m = m0 + u T (u < G) per pass over the taps, each tap read once per G
// multiply-add pairs, and stores u[m] e^{-j w m D} into s (padded index).
// FIR + decimate (Eq. 8-10, polyphase): output m sums, over the phase rows
// p, g[J - p - D c] xs[p rs + m + c] for c = 0 .. n_p - 1 (tap k = J - q,
// q = p + D c), then takes the rotation of the mix.  A thread computes B
// adjacent outputs, which read the same row window shifted by one sample: a
// window of B samples slides along the row in registers, so each tap costs
// one shared-memory read instead of B.  B = 3 keeps the threads' reads and
// stores (stride B) on distinct banks.  A block that runs past L_out reads at
// most up to index D rs (the FFT area, inside the allocation); its results
// are discarded.
template <int B, int T>
__device__ __forceinline__ void zoom_fir_blocked(const float4* tap, const float* xs, float2* s, int n_taps,
                                                 int lout, int rs, uint64_t Cn, int D, int t) {
    const int J = n_taps - 1;
    const float2 step = unit_fixed(Cn * (uint64_t)D, true);     // e^{-j w D}
    for (int m0 = B * t; m0 < lout; m0 += B * T) {
        float re[B], im[B];
#pragma unroll
        for (int u = 0; u < B; ++u) re[u] = im[u] = 0.f;
        for (int p = 0; p < D && p <= J; ++p) {
            const float* row = xs + p * rs + m0;
            const float4* tp = tap + (J - p);                // tap of step c: tp[-D c]
            const int np = (J - p) / D + 1;
            float w[B];
#pragma unroll
            for (int u = 0; u + 1 < B; ++u) w[u + 1] = row[u];
#pragma unroll 3
            for (int c = 0; c < np; ++c) {
#pragma unroll
                for (int u = 0; u + 1 < B; ++u) w[u] = w[u + 1];
                w[B - 1] = row[c + B - 1];                   // window: w[u] = row[c + u]
                const float4 g = tp[-D * c];
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    re[u] = fmaf(g.x, w[u], re[u]);
                    im[u] = fmaf(g.y, w[u], im[u]);
                }
            }
        }
        // e^{-j w m D} for m = m0 .. m0 + B - 1: the first from the exact
        // phase, the next by the one-output step (B - 1 products)
        float2 rot = unit_fixed(Cn * ((uint64_t)m0 * (uint64_t)D), true);
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int m = m0 + u;
            if (m < lout) s[pidx(m)] = cmul(make_float2(re[u], im[u]), rot);
            if (u + 1 < B) rot = cmul(rot, step);
        }
    }
}

// LO4: the launch guarantees L_out <= 4 T, so only the first four FFT inputs
// of a thread can be nonzero (BlockFFT::run_lo4); a separate instance, since
// both FFT forms in one kernel spill at 64 registers.
template <int K, bool LO4 = false>
__global__ void __launch_bounds__(FFTShape<K>::T, FFTShape<K>::T >= 1024 ? 1 : (FFTShape<K>::T >= 32 ? 1024 / FFTShape<K>::T : 32)) k_zoom(ZoomArgs a) {
    using FFT = BlockFFT<K, false>;
    constexpr int E = FFT::E, T = FFT::T;
    extern __shared__ float4 smem4[];
    const int t = threadIdx.x;
    const int64_t b = blockIdx.x;
    int n = a.n, n_taps = a.n_taps, D = a.d, logd = a.logd, lout = a.lout, rs = a.rs;
    uint64_t Cn = a.Cn;
    const float* taps = a.taps;
    int64_t xo = b * a.ld_x, Xo = b * a.ld_X;
    if (a.items) {
        const RaggedItem& it = a.items[b];
        xo = it.x_off;
        Xo = it.out_off;
        n = it.n;
        n_taps = it.n_taps;
        D = it.d;
        logd = is_pow2_dev(D) ? ilog2c(D) : -1;
        lout = it.lout;
        rs = it.rs;
        Cn = it.A;
        taps = a.taps + it.tab_off;
    }
    const int J = n_taps - 1;

    // shared layout: taps {g.re, g.im, offset} | polyphase x | FFT exchange
    // (the decimated u[m] is staged in the FFT exchange area)
    float4* tap = smem4;
    float* xs = reinterpret_cast<float*>(smem4 + n_taps);
    float2* s = reinterpret_cast<float2*>(smem4 + n_taps) + (D * rs + 1) / 2;

    // complex taps g[k] = h[k] e^{+j 2 pi c k} and their polyphase offsets
    for (int k = t; k < n_taps; k += T) {
        const float h = __ldg(taps + k);
        const float2 e = unit_fixed(Cn * (uint64_t)k, false);
        const int q = J - k;
        const int off = (q % D) * rs + q / D;
        tap[k] = make_float4(h * e.x, h * e.y, __int_as_float(off), 0.f);
    }
    // extended trace xe[j] = x[j - J] (zero outside [0, N)), by phase
    const float* xr = a.x + xo;
    const int total = D * rs;
    if (logd >= 2 && (n & 3) == 0 && (reinterpret_cast<uintptr_t>(xr) & 15) == 0) {
        // 16-byte loads of four samples; the zeros before and after the trace
        // separately (j + 4 q: the warp's stores of one sample index fall in
        // one phase row at most two rows, consecutive columns)
        const int dm = D - 1;
        for (int j = t; j < J; j += T) xs[(j & dm) * rs + (j >> logd)] = 0.f;
        for (int j = J + n + t; j < total; j += T) xs[(j & dm) * rs + (j >> logd)] = 0.f;
        const float4* x4 = reinterpret_cast<const float4*>(xr);
        for (int q = t; q < (n >> 2); q += T) {
            const float4 x = __ldg(x4 + q);
            const int j = 4 * q + J;
            xs[(j & dm) * rs + (j >> logd)] = x.x;
            xs[((j + 1) & dm) * rs + ((j + 1) >> logd)] = x.y;
            xs[((j + 2) & dm) * rs + ((j + 2) >> logd)] = x.z;
            xs[((j + 3) & dm) * rs + ((j + 3) >> logd)] = x.w;
        }
    } else if (logd >= 0) {
        const int dm = D - 1;
        for (int j = t; j < total; j += T) {
            const int src = j - J;
            const float xv = (src >= 0 && src < n) ? __ldg(xr + src) : 0.f;
            xs[(j & dm) * rs + (j >> logd)] = xv;
        }
    } else {
        for (int j = t; j < total; j += T) {
            const int src = j - J;
            const float xv = (src >= 0 && src < n) ? __ldg(xr + src) : 0.f;
            xs[(j % D) * rs + j / D] = xv;
        }
    }
    __syncthreads();

    zoom_fir_blocked<3, T>(tap, xs, s, n_taps, lout, rs, Cn, D, t);
    __syncthreads();
    float2 v[E];
    if constexpr (LO4) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = t + T * i;
            v[i] = m < lout ? s[pidx(m)] : make_float2(0.f, 0.f);
        }
        FFT::run_lo4(v, s, t, a.tw);
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int m = t + T * i;
            v[i] = m < lout ? s[pidx(m)] : make_float2(0.f, 0.f);
        }
        FFT::run(v, s, t, a.tw);
    }
    float2* Xr = a.X + Xo;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int j = t + T * i;
        Xr[(j + K / 2) & (K - 1)] = v[i];
    }
}

// The blocked FIR of zoom_fir_blocked on two traces side by side: xs holds
// (trace 2p, trace 2p+1) sample pairs, taps are stored (g.re, g.re, g.im,
// g.im), and every accumulator is a packed pair.  The window reads of a warp
// (float2 at stride B = 3) and its staging stores fall on distinct banks.
template <int B, int T>
__device__ __forceinline__ void zoom_fir_blocked2(const float4* tap, const float2* xs, float4* s, int n_taps,
                                                  int lout, int rs, uint64_t Cn, int D, int t) {
    const int J = n_taps - 1;
    const float2 step = unit_fixed(Cn * (uint64_t)D, true);     // e^{-j w D}
    for (int m0 = B * t; m0 < lout; m0 += B * T) {
        float2 re[B], im[B];
#pragma unroll
        for (int u = 0; u < B; ++u) re[u] = im[u] = make_float2(0.f, 0.f);
        for (int p = 0; p < D && p <= J; ++p) {
            const float2* row = xs + p * rs + m0;
            const float4* tp = tap + (J - p);                // tap of step c: tp[-D c]
            const int np = (J - p) / D + 1;
            float2 w[B];
#pragma unroll
            for (int u = 0; u + 1 < B; ++u) w[u + 1] = row[u];
#pragma unroll 3
            for (int c = 0; c < np; ++c) {
#pragma unroll
                for (int u = 0; u + 1 < B; ++u) w[u] = w[u + 1];
                w[B - 1] = row[c + B - 1];                   // window: w[u] = row[c + u]
                const float4 g = tp[-D * c];
                const float2 gr = make_float2(g.x, g.y), gi = make_float2(g.z, g.w);
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    re[u] = fma2(gr, w[u], re[u]);
                    im[u] = fma2(gi, w[u], im[u]);
                }
            }
        }
        float2 rot = unit_fixed(Cn * ((uint64_t)m0 * (uint64_t)D), true);
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int m = m0 + u;
            if (m < lout) sts(s, pidx(m), mul_tw<false>(C2{re[u], im[u]}, rot));
            if (u + 1 < B) rot = cmul(rot, step);
        }
    }
}

// Two-lane variant: traces 2p and 2p+1 share one CTA.  Their samples sit
// side by side in shared memory (one float2 per polyphase slot), so each tap
// -- stored duplicated as (g.re, g.re, g.im, g.im) -- feeds both traces with
// two packed multiply-adds, and the FFT runs on packed pairs.
template <int K>
__global__ void __launch_bounds__(FFTShape<K>::T, FFTShape<K>::T >= 512 ? 1 : FFTShape<K>::T >= 128 ? 512 / FFTShape<K>::T : 4)
    k_zoom2(ZoomArgs a) {
    using FFT = BlockFFT<K, false, C2>;
    constexpr int E = FFT::E, T = FFT::T;
    extern __shared__ float4 smem4[];
    const int t = threadIdx.x;
    const int64_t b0 = 2 * (int64_t)blockIdx.x, b1 = b0 + 1;
    const bool live1 = b1 < a.batch;
    const int D = a.d;

    // shared layout: taps (g.re, g.re, g.im, g.im) | polyphase x pairs |
    // FFT exchange (float4) | slack (a window that runs past L_out reads into
    // the FFT area; its results are discarded)
    float4* tap = smem4;
    float2* xs = reinterpret_cast<float2*>(smem4 + a.n_taps);
    float4* s = smem4 + a.n_taps + (D * a.rs + 1) / 2;

    for (int k = t; k < a.n_taps; k += T) {
        const float h = __ldg(a.taps + k);
        const float2 e = unit_fixed(a.Cn * (uint64_t)k, false);
        tap[k] = make_float4(h * e.x, h * e.x, h * e.y, h * e.y);
    }
    const int J = a.n_taps - 1;
    const float* x0 = a.x + b0 * a.ld_x;
    const float* x1 = a.x + (live1 ? b1 : b0) * a.ld_x;
    const int total = D * a.rs;
    for (int j = t; j < total; j += T) {
        const int src = j - J;
        const bool in = src >= 0 && src < a.n;
        const float2 xv = make_float2(in ? __ldg(x0 + src) : 0.f, (in && live1) ? __ldg(x1 + src) : 0.f);
        const int slot = a.logd >= 0 ? (j & (D - 1)) * a.rs + (j >> a.logd) : (j % D) * a.rs + j / D;
        xs[slot] = xv;
    }
    __syncthreads();

    // FIR + decimate for both traces at once: the blocked sliding window of
    // zoom_fir_blocked with packed (trace 2p, trace 2p+1) samples, so each
    // tap read feeds 2 B outputs with B packed multiply-adds per component
    zoom_fir_blocked2<3, T>(tap, xs, s, a.n_taps, a.lout, a.rs, a.Cn, D, t);
    __syncthreads();
    C2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int m = t + T * i;
        v[i] = m < a.lout ? lds(s, pidx(m), (C2*)nullptr) : C2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    }
    FFT::run(v, s, t, a.tw);
    float2* X0 = a.X + b0 * a.ld_X;
    float2* X1 = a.X + (live1 ? b1 : b0) * a.ld_X;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int j = (t + T * i + K / 2) & (K - 1);
        X0[j] = lane_a(v[i]);
        if (live1) X1[j] = lane_b(v[i]);
    }
}

// ---------------------------------------------------------------------------
// Large Zoom FFTs (a long trace, or N_FFT/D above one CTA): the FIR-decimate
// step runs here, kFirChunk kept outputs per CTA and many CTAs per trace, and
// writes u[m] (mix and rotation applied) to a workspace; the K-point FFT and
// the ascending-frequency store follow in the pruned cluster FFT
// (k_fft_c2c_pruned).  Same arithmetic as k_zoom.
constexpr int kFirChunk = 256;

struct FirArgs {
    const float* x;
    int64_t batch;
    int n;
    int64_t ld_x;
    const float* taps;
    int n_taps, d, logd, lout, rs, chunks;
    uint64_t Cn;
    float2* u;
    int64_t ld_u;
    const RaggedItem* items;   // ragged batch (else null)
};

__global__ void __launch_bounds__(kFirChunk) k_zoom_fir(FirArgs a) {
    extern __shared__ float4 smem4[];
    const int t = threadIdx.x;
    const int64_t b = blockIdx.x / a.chunks;
    const int m0 = (int)(blockIdx.x % a.chunks) * kFirChunk;
    int n = a.n, n_taps = a.n_taps, D = a.d, logd = a.logd, lout = a.lout, rs = a.rs;
    uint64_t Cn = a.Cn;
    const float* taps = a.taps;
    int64_t xo = b * a.ld_x, uo = b * a.ld_u;
    if (a.items) {
        const RaggedItem& it = a.items[b];
        xo = it.x_off;
        uo = it.u_off;
        n = it.n;
        n_taps = it.n_taps;
        D = it.d;
        logd = is_pow2_dev(D) ? ilog2c(D) : -1;
        lout = it.lout;
        rs = kFirChunk + (n_taps - 1) / D + 2;
        rs += (rs & 1) ^ 1;
        Cn = it.A;
        taps = a.taps + it.tab_off;
        if (m0 >= lout) return;            // this trace has fewer chunks (whole CTA)
    }
    const int J = n_taps - 1;
    float4* tap = smem4;
    float* xs = reinterpret_cast<float*>(smem4 + n_taps);

    for (int k = t; k < n_taps; k += kFirChunk) {
        const float h = __ldg(taps + k);
        const float2 e = unit_fixed(Cn * (uint64_t)k, false);
        const int q = J - k;
        tap[k] = make_float4(h * e.x, h * e.y, __int_as_float((q % D) * rs + q / D), 0.f);
    }
    // window of the extended trace for outputs m0 .. m0 + kFirChunk - 1:
    // local index jj = j - m0 D, sample x[j - J]
    const float* xr = a.x + xo;
    const int total = D * rs;
    const int64_t base = (int64_t)m0 * D - J;
    for (int jj = t; jj < total; jj += kFirChunk) {
        const int64_t src = base + jj;
        const float xv = (src >= 0 && src < n) ? __ldg(xr + src) : 0.f;
        const int slot = logd >= 0 ? (jj & (D - 1)) * rs + (jj >> logd) : (jj % D) * rs + jj / D;
        xs[slot] = xv;
    }
    __syncthreads();
    const int m = m0 + t;
    if (m < lout) {
        float re = 0.f, im = 0.f;
        const float* xm = xs + t;
        for (int k = 0; k < n_taps; ++k) {
            const float4 g = tap[k];
            const float xv = xm[__float_as_int(g.z)];
            re = fmaf(g.x, xv, re);
            im = fmaf(g.y, xv, im);
        }
        const float2 rot = unit_fixed(Cn * ((uint64_t)m * (uint64_t)D), true);
        a.u[uo + m] = cmul(make_float2(re, im), rot);
    }
}

bool zoom_big_plan(int64_t batch, int64_t n, int64_t d, int64_t n_taps, int64_t n_fft, double fs, double f1,
                   double f2, ZoomPlan* p, std::string* why) {
    *p = ZoomPlan();
    const int64_t K = n_fft / d;
    const int64_t lout = (n + n_taps - 1 + d - 1) / d;
    int64_t rs = kFirChunk + (n_taps - 1) / d + 2;
    if ((rs & 1) == 0) ++rs;
    const size_t smem = (size_t)n_taps * 16 + (size_t)d * rs * 4;
    if (smem > 200 * 1024) {
        *why = "zoom: taps and decimation too large for the FIR tile";
        return false;
    }
    FftPlan fp;
    if (!c2c_plan(batch, lout, K, &fp, why)) return false;
    p->n = (int)n; p->d = (int)d; p->n_taps = (int)n_taps; p->K = (int)K; p->lout = (int)lout;
    p->rs = (int)rs;
    p->Cn = cycles_to_fixed(0.5 * (f1 + f2) / fs);
    p->threads = kFirChunk;
    p->smem = smem;
    p->big = true;
    p->fft = fp;
    return true;
}

cudaError_t zoom_big_launch(const ZoomPlan& p, const float* x, int64_t batch, int64_t ld_x, const float* taps,
                            float2* work, const float2* tw, const float2* tab, float2* X, int64_t ld_X,
                            cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    FirArgs a = {};
    a.x = x; a.batch = batch; a.n = p.n; a.ld_x = ld_x; a.taps = taps;
    a.n_taps = p.n_taps; a.d = p.d; a.logd = is_pow2(p.d) ? ilog2(p.d) : -1; a.lout = p.lout; a.rs = p.rs;
    a.chunks = (p.lout + kFirChunk - 1) / kFirChunk; a.Cn = p.Cn;
    a.u = work; a.ld_u = p.fft.LZ;
    cudaError_t e = cudaFuncSetAttribute(k_zoom_fir, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    k_zoom_fir<<<(unsigned)(batch * a.chunks), kFirChunk, p.smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return c2c_launch(p.fft, work, p.fft.LZ, p.lout, batch, p.K / 2, tw, tab, X, ld_X, st);
}

using ZoomKernel = void (*)(ZoomArgs);

static ZoomKernel zoom_kernel2_for(int K) {
    switch (K) {
        case 16: return k_zoom2<16>;
        case 32: return k_zoom2<32>;
        case 64: return k_zoom2<64>;
        case 128: return k_zoom2<128>;
        case 256: return k_zoom2<256>;
        case 512: return k_zoom2<512>;
        case 1024: return k_zoom2<1024>;
        case 2048: return k_zoom2<2048>;
        case 4096: return k_zoom2<4096>;
        case 8192: return k_zoom2<8192>;
        default: return nullptr;
    }
}

static ZoomKernel zoom_kernel_for(int K, bool lo4 = false) {
    if (lo4) {
        switch (K) {
            case 512: return k_zoom<512, true>;
            case 1024: return k_zoom<1024, true>;
            case 2048: return k_zoom<2048, true>;
            case 4096: return k_zoom<4096, true>;
            case 8192: return k_zoom<8192, true>;
            case 16384: return k_zoom<16384, true>;
            default: break;
        }
    }
    switch (K) {
        case 1: return k_zoom<1>;
        case 2: return k_zoom<2>;
        case 4: return k_zoom<4>;
        case 8: return k_zoom<8>;
        case 16: return k_zoom<16>;
        case 32: return k_zoom<32>;
        case 64: return k_zoom<64>;
        case 128: return k_zoom<128>;
        case 256: return k_zoom<256>;
        case 512: return k_zoom<512>;
        case 1024: return k_zoom<1024>;
        case 2048: return k_zoom<2048>;
        case 4096: return k_zoom<4096>;
        case 8192: return k_zoom<8192>;
        case 16384: return k_zoom<16384>;
        default: return nullptr;
    }
}

bool zoom_plan(int64_t n, int64_t d, int64_t n_taps, int64_t n_fft, double fs, double f1,
               double f2, ZoomPlan* p, std::string* why) {
    *p = ZoomPlan();
    const int64_t K = n_fft / d;
    const int64_t lout = (n + n_taps - 1 + d - 1) / d;
    if (K > 16384) {
        *why = "zoom: N_FFT/D above 16384 needs the multi-pass path";
        return false;
    }
    const int E = K < 16 ? (int)K : 16;
    const int T = (int)(K / E);
    // Row p holds columns 0 .. rs-1; kept outputs read columns up to
    // (L_out - 1) + (L_h - 1)/D.  The last group of four outputs per thread
    // may run past L_out: those reads (results discarded) stay inside the
    // allocation, in the FFT area after the rows plus kZoomGroup T floats of
    // slack at the end.
    const int64_t rs = zoom_rows(lout, n_taps, d);
    const size_t smem = (size_t)n_taps * 16 + (size_t)((d * rs + 1) / 2) * 8 +
                        (size_t)padded_len((int)K) * 8 + (size_t)kZoomGroup * T * 4;
    if (smem > 200 * 1024) {
        *why = "zoom: trace plus taps exceed one CTA's shared memory; needs the multi-pass path";
        return false;
    }
    p->n = (int)n; p->d = (int)d; p->n_taps = (int)n_taps; p->K = (int)K; p->lout = (int)lout;
    p->rs = (int)rs;
    // two-lane layout: taps (16 B) + polyphase pairs + float4 FFT area + slack
    p->smem2 = (size_t)n_taps * 16 + (size_t)((d * rs + 1) / 2) * 16 + (size_t)padded_len((int)K) * 16 +
               (size_t)kZoomGroup * T * 8;
    p->dual = K >= 16 && K <= 8192 && p->smem2 <= 200 * 1024;
    p->Cn = cycles_to_fixed(0.5 * (f1 + f2) / fs);
    p->threads = T;
    p->smem = smem;
    return true;
}

cudaError_t zoom_launch(const ZoomPlan& p, const float* x, int64_t batch, int64_t ld_x,
                        const float* taps, const float2* tw, float2* X, int64_t ld_X, cudaStream_t st,
                        int lanes) {
    if (batch == 0) return cudaSuccess;
    const bool dual = p.dual && batch >= 2 && lanes != 1;
    // L_out <= 4 T (T = K/16): the FFT's first pass sees four inputs per thread
    ZoomKernel k = dual ? zoom_kernel2_for(p.K) : zoom_kernel_for(p.K, (int64_t)p.lout * 4 <= p.K);
    if (!k) return cudaErrorInvalidValue;
    const size_t smem = dual ? p.smem2 : p.smem;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ZoomArgs a = {};
    a.x = x; a.batch = batch; a.n = p.n; a.ld_x = ld_x; a.taps = taps;
    a.n_taps = p.n_taps; a.d = p.d; a.logd = is_pow2(p.d) ? ilog2(p.d) : -1;
    a.lout = p.lout; a.rs = p.rs; a.Cn = p.Cn; a.tw = tw;
    a.X = X; a.ld_X = ld_X;
    const int64_t grid = dual ? (batch + 1) / 2 : batch;
    k<<<(unsigned)grid, p.threads, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Ragged batches (per-trace parameters from RaggedItem).

// Row stride of the polyphase layout: at least the columns a kept output
// reads, (L_out - 1) + (L_h - 1)/D + 2.  A warp stages 32 consecutive samples,
// D phases x 32/D columns; for D a power of two up to 32 the stride is m mod
// 2m (m = 32/D), so the D rows start m banks apart and the warp's stores hit
// 32 different banks.  Otherwise (and for D = 1) the stride is odd.
int zoom_rows(int64_t lout, int64_t n_taps, int64_t d) {
    const int64_t need = (lout - 1) + (n_taps - 1) / d + 2;
    if (d >= 2 && d <= 32 && is_pow2(d)) {
        const int64_t m = 32 / d;
        return (int)(need + ((m - need % (2 * m)) % (2 * m) + 2 * m) % (2 * m));
    }
    return (int)(need | 1);
}

size_t zoom_smem_for(int n_taps, int d, int rs, int K) {
    const int E = K < 16 ? K : 16;
    const int T = K / E;
    return (size_t)n_taps * 16 + (size_t)((d * rs + 1) / 2) * 8 + (size_t)padded_len(K) * 8 +
           (size_t)kZoomGroup * T * 4;
}

int fir_rows(int64_t n_taps, int64_t d) {
    int64_t rs = kFirChunk + (n_taps - 1) / d + 2;
    return (int)(rs | 1);
}

size_t fir_smem_for(int n_taps, int d) { return (size_t)n_taps * 16 + (size_t)d * fir_rows(n_taps, d) * 4; }

int fir_chunk() { return kFirChunk; }

cudaError_t zoom_ragged_launch(int K, const RaggedItem* items, int64_t count, size_t smem, const float* x_pool,
                               const float* taps_pool, const float2* tw, float2* X_pool, cudaStream_t st, bool lo4) {
    if (count == 0) return cudaSuccess;
    ZoomKernel k = zoom_kernel_for(K, lo4);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ZoomArgs a = {};
    a.x = x_pool; a.batch = count; a.taps = taps_pool; a.tw = tw; a.X = X_pool; a.items = items;
    const int E = K < 16 ? K : 16;
    k<<<(unsigned)count, K / E, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t zoom_fir_ragged_launch(const RaggedItem* items, int64_t count, int chunks_max, size_t smem,
                                   const float* x_pool, const float* taps_pool, float2* work, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_zoom_fir, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    FirArgs a = {};
    a.x = x_pool; a.batch = count; a.taps = taps_pool; a.chunks = chunks_max; a.u = work; a.items = items;
    k_zoom_fir<<<(unsigned)(count * chunks_max), kFirChunk, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Ragged batches as one persistent launch (work queue): every trace has its
// own N, D, taps and K = N_FFT/D <= 16384.  A unit holds up to 16384/K traces
// of one K on a 1024-thread CTA, each trace on K/16 threads with its own
// slice of shared memory (taps, polyphase trace, FFT area: the k_zoom
// layout).  Where the slices of 16384/K traces do not fit, the unit holds F
// fewer traces and the remaining thread groups run the FFT's barriers on a
// scratch FFT area, touching nothing else.  Units (largest K first) are
// popped from an atomic counter by persistent CTAs, one per SM.
struct ZoomQueueArgs {
    const RaggedItem* items;
    const ZoomUnit* units;
    int nunits;
    unsigned* counter;
    const float* x;
    const float* taps;
    float2* X;
    const float2* tw;          // BlockFFT twiddles of every size (radix-16 layout)
};

constexpr int kZoomQueueThreads = 1024;

template <int K>
__device__ __forceinline__ void zoom_queue_unit(const ZoomQueueArgs& a, const ZoomUnit& u, unsigned char* smem) {
    using FFT = BlockFFT<K, false>;
    constexpr int E = FFT::E, T = FFT::T;
    const int f = threadIdx.x / T;
    const int t = threadIdx.x - f * T;
    const bool live = f < u.count;                     // u.count <= u.F
    const RaggedItem it = a.items[u.first + (live ? f : 0)];
    const int n = it.n, n_taps = it.n_taps, D = it.d, lout = it.lout, rs = it.rs;
    const int logd = is_pow2_dev(D) ? ilog2c(D) : -1;
    const uint64_t Cn = it.A;
    const int J = n_taps - 1;
    float4* slice = reinterpret_cast<float4*>(smem + (size_t)(f < u.F ? f : 0) * u.slice);
    float4* tap = slice;
    float* xs = reinterpret_cast<float*>(slice + n_taps);
    float2* s = live ? reinterpret_cast<float2*>(slice + n_taps) + (D * rs + 1) / 2
                     : reinterpret_cast<float2*>(smem + u.scratch);
    if (live) {
        const float* taps = a.taps + it.tab_off;
        for (int k = t; k < n_taps; k += T) {
            const float h = __ldg(taps + k);
            const float2 e = unit_fixed(Cn * (uint64_t)k, false);
            const int q = J - k;
            tap[k] = make_float4(h * e.x, h * e.y, __int_as_float((q % D) * rs + q / D), 0.f);
        }
        const float* xr = a.x + it.x_off;
        const int total = D * rs;
        for (int j = t; j < total; j += T) {
            const int src = j - J;
            const float xv = (src >= 0 && src < n) ? __ldg(xr + src) : 0.f;
            const int slot = logd >= 0 ? (j & (D - 1)) * rs + (j >> logd) : (j % D) * rs + j / D;
            xs[slot] = xv;
        }
    }
    __syncthreads();
    if (live) zoom_fir_blocked<3, T>(tap, xs, s, n_taps, lout, rs, Cn, D, t);
    __syncthreads();
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int m = t + T * i;
        v[i] = (live && m < lout) ? s[pidx(m)] : make_float2(0.f, 0.f);
    }
    FFT::run(v, s, t, a.tw + (K <= 16 ? 0 : fft_twiddle_offset(K)));
    if (!live) return;
    float2* Xr = a.X + it.out_off;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int j = t + T * i;
        Xr[(j + K / 2) & (K - 1)] = v[i];
    }
}

__global__ void __launch_bounds__(kZoomQueueThreads, 1) k_zoom_queue(ZoomQueueArgs a) {
    extern __shared__ float4 smem4[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem4);
    __shared__ int s_unit;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_unit = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int ui = s_unit;
        if (ui >= a.nunits) return;
        const ZoomUnit u = a.units[ui];
        switch (u.K) {
            case 64: zoom_queue_unit<64>(a, u, smem); break;
            case 128: zoom_queue_unit<128>(a, u, smem); break;
            case 256: zoom_queue_unit<256>(a, u, smem); break;
            case 512: zoom_queue_unit<512>(a, u, smem); break;
            case 1024: zoom_queue_unit<1024>(a, u, smem); break;
            case 2048: zoom_queue_unit<2048>(a, u, smem); break;
            case 4096: zoom_queue_unit<4096>(a, u, smem); break;
            case 8192: zoom_queue_unit<8192>(a, u, smem); break;
            default: zoom_queue_unit<16384>(a, u, smem); break;
        }
    }
}

int zoom_queue_groups(int K) { return kZoomQueueThreads / (K / 16); }

cudaError_t zoom_queue_launch(const RaggedItem* items, const ZoomUnit* units, int nunits, unsigned* counter,
                              size_t smem, const float* x_pool, const float* taps_pool, const float2* tw,
                              float2* X_pool, int ctas, cudaStream_t st) {
    if (nunits == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_zoom_queue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ZoomQueueArgs a = {};
    a.items = items; a.units = units; a.nunits = nunits; a.counter = counter;
    a.x = x_pool; a.taps = taps_pool; a.X = X_pool; a.tw = tw;
    k_zoom_queue<<<(unsigned)std::max(1, std::min(ctas, nunits)), kZoomQueueThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace spec
