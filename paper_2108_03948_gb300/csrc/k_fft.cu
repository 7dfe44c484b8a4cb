// k_fft.cu -- zero-padded FFT of real traces (Section 2.1, Eq. 2-3 and the
// zero-padding paragraph): X[k] = sum_{n<N} x[n] e^{-j 2 pi k n/N_FFT},
// k = 0 .. N_FFT/2.
//
// Method (one launch, one HBM read of x and one write of X):
//  1. pack pairs of real samples, z[m] = x[2m] + j x[2m+1], m < ceil(N/2),
//     a complex sequence of H = N_FFT/2 points of which only LZ are nonzero;
//  2. prune the padding: bin R q + r of the H-point FFT equals bin q of the
//     LZ-point FFT of z[m] w_H^{r m} (R = H/LZ residues), so R dense LZ-point
//     FFTs replace the sparse H-point one;
//  3. unpack: X[k] = (Z[k] + conj Z[H-k])/2 - j/2 w^k (Z[k] - conj Z[H-k]),
//     w = e^{-j 2 pi/N_FFT}, for the pair (k, H - k) at once.
// Each CTA holds <= 8192 complex points; a trace that needs more is spread
// over a thread-block cluster.  Step 3 reads Z in natural order from shared
// memory; in a cluster each CTA owns a contiguous chunk of Z and the others
// reach it through distributed shared memory.  All twiddles come from tables
// generated once in float64.
#include <cooperative_groups.h>

#include <cstdlib>

#include "fft_block.cuh"
#include "mbarrier.cuh"
#include "spec_internal.h"

namespace cg = cooperative_groups;

namespace spec {

struct FftArgs {
    const float* x;
    int64_t batch;
    int n;
    int64_t ld_x;
    int H, logR, Rc, C, F, logChunk, trace_smem;
    const float2* tw;     // BlockFFT<LZ> twiddles
    const float2* tab;    // [w_H^{r t}: R x T][w_H^{r T i}: R x E][w_{2H}^k: H/2 + 1]
    float2* X;
    int64_t ld_X;
    const RaggedItem* items;   // ragged batch: per-trace x / X offsets and n (else null)
    int paired;                // C > 1 without a cluster: each CTA owns residue pairs {r, R - r}
    unsigned* status;          // bounded waits (persistent forms): the context's status word
    uint64_t timeout_ns;
};

// Residue of local FFT rl in CTA `rank` of a trace.  Contiguous by default.
// With `paired` (no cluster), CTA c owns a run of g = Rc/2 consecutive
// residues c g .. c g + g - 1 (local 0 .. g-1) and their mirrors R - r
// (local g .. 2g-1; CTA 0 holds 0 and R/2, both their own mirrors), so every
// partner Z[H - k] of its Z[k] is local and its outputs form runs of g.
__device__ __forceinline__ int residue_of(const FftArgs& a, int rank, int rl) {
    if (!a.paired) return rank * a.Rc + rl;
    if (a.Rc == 1) return rank;                                   // R = 2: both residues self-paired
    const int R = 1 << a.logR;
    const int g = a.Rc >> 1;
    if (rl < g) return rank * g + rl;
    const int j = rl - g;
    return (rank == 0 && j == 0) ? R / 2 : R - (rank * g + j);
}

// Cluster staging for the unpack.  CTA c of a cluster of C unpacks the pairs
// k in [c P, c P + P), P = H/(2C) (the last CTA also k = H/2), so it receives
// exactly the values those pairs read: Z[k] at slot k - c P (0 .. P) and
// Z[H - k] at slot P + 1 + (k - c P).  Every value crosses the cluster once,
// as a remote store; the unpack then reads only its own shared memory.
__device__ __forceinline__ int2 pair_home(int j, int H, int logP, int C) {
    const int half = H >> 1;
    if (j <= half) {
        const int c = min(j >> logP, C - 1);
        return make_int2(c, j - (c << logP));
    }
    const int kk = H - j;
    const int c = kk >> logP;
    return make_int2(c, (1 << logP) + 1 + kk - (c << logP));
}

// Store v at element `idx` of the same shared array in CTA `cta` of the
// cluster (distributed shared memory through the shared-memory path).
__device__ __forceinline__ void dsmem_store(float2* local_base, int idx, unsigned cta, float2 v) {
    const uint32_t local = (uint32_t)__cvta_generic_to_shared(local_base + idx);
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(cta));
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(remote), "f"(v.x), "f"(v.y) : "memory");
}

// Cluster barrier whose arrival does not order this thread's memory accesses
// (used where only the completion of already-consumed reads matters).
__device__ __forceinline__ void cluster_arrive_relaxed_wait() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// X[k] and X[H - k] from A = Z[k], B = Z[H - k] (Section 2.1 real-input unpack)
__device__ __forceinline__ void unpack_pair(float2* Xr, int k, int H, float2 A, float2 B, float2 w) {
    const float2 sp = mul2(make_float2(A.x + B.x, A.y - B.y), make_float2(0.5f, 0.5f));
    const float2 dm = mul2(make_float2(A.x - B.x, A.y + B.y), make_float2(0.5f, 0.5f));
    const float2 wd = cmul(w, dm);
    Xr[k] = make_float2(sp.x + wd.y, sp.y - wd.x);
    if (H - k != k) Xr[H - k] = make_float2(sp.x - wd.y, -sp.y - wd.x);
}

// Packed input of one residue FFT, pre-twiddled: v[i] = z[m] w_H^{r m},
// z[m] = x[2m] + j x[2m+1], m = t + T i, the twiddle w_H^{r t} w_H^{r T i}.
template <int E, int T>
__device__ __forceinline__ void load_pretwiddled(float2 (&v)[E], const float* xr, int n, bool live,
                                                 const float2* wt_p, const float2* wi_p, int t) {
    const float2 wt = __ldg(wt_p);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int m = t + T * i;
        float re = 0.f, im = 0.f;
        if (live && 2 * m < n) re = __ldg(xr + 2 * m);
        if (live && 2 * m + 1 < n) im = __ldg(xr + 2 * m + 1);
        v[i] = cmul(make_float2(re, im), cmul(wt, __ldg(wi_p + i)));
    }
}

__device__ __forceinline__ unsigned opaque_tid() {
    unsigned v;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(v));
    return v;
}
__device__ __forceinline__ unsigned opaque_ctaid() {
    unsigned v;
    asm volatile("mov.u32 %0, %%ctaid.x;" : "=r"(v));
    return v;
}

template <int E, int T>
__device__ __forceinline__ void epilogue(const FftArgs& a, float2 (&v)[E]);

template <int LZ, int EMAX>
__global__ void __launch_bounds__(EMAX == 32 ? 256 : 1024, EMAX == 32 ? 2 : 1) k_fft_real_padded(FftArgs a) {
    using FFT = BlockFFT<LZ, false, float2, EMAX>;
    constexpr int E = FFT::E;
    constexpr int T = FFT::T;
    extern __shared__ float2 smem[];

    const int per_trace = a.Rc * T;
    const int tid = threadIdx.x;
    const int f = tid / per_trace;
    const int lt = tid - f * per_trace;          // thread index within the trace
    const int rl = lt / T;
    const int t = lt - rl * T;
    const int rank = a.C > 1 ? (int)(blockIdx.x % a.C) : 0;
    const int64_t b = (int64_t)(blockIdx.x / a.C) * a.F + f;
    const bool live = b < a.batch;
    int n = a.n;
    int64_t xo = (live ? b : 0) * a.ld_x;
    if (a.items && live) {
        const RaggedItem& it = a.items[b];
        xo = it.x_off;
        n = it.n;
    }
    const int R = 1 << a.logR;
    const int r = residue_of(a, rank, rl);       // residue of this thread's FFT
    float2* zs = smem + f * a.trace_smem;        // this trace's shared memory
    float2* s = zs + rl * padded_len(LZ);

    // 1-2. packed, pre-twiddled input: v[i] = z[m] w_H^{r m}, m = t + T i.
    float2 v[E];
    load_pretwiddled<E, T>(v, a.x + xo, n, live, a.tab + r * T + t, a.tab + R * T + r * E, t);
    FFT::run(v, s, t, a.tw);
    // From here on, the thread's placement is derived again from fresh reads
    // of its indices (opaque to the compiler), so that only v[] is live
    // across the FFT (register pressure at 64 registers).
    epilogue<E, T>(a, v);
}

// Unpack of a CTA that owns residue pairs (no cluster): each residue's Z in
// natural order in its own shared region, then every output pair (k, H - k)
// with k in its residues from local values.  X is written at stride R.
template <int E, int T>
__device__ __forceinline__ void paired_unpack(const FftArgs& a, float2 (&v)[E], float2* zs, int rl, int t, int lt,
                                              int per_trace, bool live, int64_t Xo) {
    constexpr int LZ = E * T;
    const int R = 1 << a.logR;
    const int H = a.H;
    __syncthreads();                                     // every FFT's exchanges are done
    float2* s = zs + rl * padded_len(LZ);
#pragma unroll
    for (int i = 0; i < E; ++i) s[pidx(t + T * i)] = v[i];
    __syncthreads();
    if (!live) return;
    float2* Xr = a.X + Xo;
    const float2* wp = a.tab + R * T + R * E;
    const int rank = a.C > 1 ? (int)(opaque_ctaid() % a.C) : 0;
    // (k, A = Z[k], B = Z[H - k]) -> X[k], X[H - k] with the twiddle of min(k, H - k)
    auto emit = [&](int k, float2 A, float2 B) {
        if (2 * k <= H) unpack_pair(Xr, k, H, A, B, __ldg(wp + k));
        else unpack_pair(Xr, H - k, H, B, A, __ldg(wp + (H - k)));
    };
    if (a.Rc == 1) {
        // R = 2: residue 0 (CTA 0) and residue 1 = R/2 (CTA 1), each its own mirror
        for (int q = lt; q <= LZ / 2; q += per_trace) {
            if (rank == 0) emit(R * q, zs[pidx(q)], zs[pidx((LZ - q) & (LZ - 1))]);
            else if (q < LZ / 2) emit(R * q + 1, zs[pidx(q)], zs[pidx(LZ - 1 - q)]);
        }
        return;
    }
    const int g = a.Rc >> 1;
    const int lg = __ffs(g) - 1;
    // the run: residue r = rank g + j (slot j) with mirror R - r (slot g + j);
    // consecutive threads take consecutive j, so X is written in runs of g
    for (int idx = lt; idx < g * LZ; idx += per_trace) {
        const int j = idx & (g - 1);
        const int q = idx >> lg;
        if (rank == 0 && j == 0) continue;                       // residue 0: below
        emit(R * q + rank * g + j, zs[j * padded_len(LZ) + pidx(q)], zs[(g + j) * padded_len(LZ) + pidx(LZ - 1 - q)]);
    }
    if (rank == 0) {
        // residue 0 (slot 0): Z[Rq] with Z[R(LZ - q)]; residue R/2 (slot g): position q with LZ-1-q
        const float2* s0 = zs;
        const float2* sh = zs + g * padded_len(LZ);
        for (int q = lt; q <= LZ / 2; q += per_trace) {
            emit(R * q, s0[pidx(q)], s0[pidx((LZ - q) & (LZ - 1))]);
            if (q < LZ / 2) emit(R * q + R / 2, sh[pidx(q)], sh[pidx(LZ - 1 - q)]);
        }
    }
}

template <int E, int T>
__device__ __forceinline__ void epilogue(const FftArgs& a, float2 (&v)[E]) {
    extern __shared__ float2 smem[];
    const int per_trace = a.Rc * T;
    const int tid = (int)opaque_tid();
    const int f = tid / per_trace;
    const int lt = tid - f * per_trace;
    const int rl = lt / T;
    const int t = lt - rl * T;
    const unsigned cta = opaque_ctaid();
    const int rank = a.C > 1 ? (int)(cta % a.C) : 0;
    const int64_t b = (int64_t)(cta / a.C) * a.F + f;
    const bool live = b < a.batch;
    const int64_t Xo = !live ? 0 : a.items ? a.items[b].out_off : b * a.ld_X;
    const int R = 1 << a.logR;
    const int r = residue_of(a, rank, rl);
    const int H = a.H;
    float2* zs = smem + f * a.trace_smem;
    if (a.paired) {
        paired_unpack<E, T>(a, v, zs, rl, t, lt, per_trace, live, Xo);
        return;
    }

    // v[i] = Z[R q + r], q = t + T i.  Every CTA of a cluster must have
    // finished its FFT (whose exchanges use this shared memory) before any of
    // them writes Z into its peers: their last exchange reads have been
    // consumed by the arithmetic before their arrival, so a relaxed arrive
    // suffices for that ordering.
    if (a.C > 1) cluster_arrive_relaxed_wait(); else __syncthreads();
    if (a.C == 1) {
#pragma unroll
        for (int i = 0; i < E; ++i) zs[pidx(((t + T * i) << a.logR) + r)] = v[i];
        __syncthreads();
    } else {
        cg::cluster_group cl = cg::this_cluster();
        const int logP = a.logChunk - 1;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int2 h = pair_home(((t + T * i) << a.logR) + r, H, logP, a.C);
            dsmem_store(zs, pidx(h.y), (unsigned)h.x, v[i]);
        }
        cl.sync();
    }

    // 3. unpack pairs (k, H - k): X[k] = (A + conj B)/2 - j/2 w (A - conj B),
    //    w = e^{-j 2 pi k/N_FFT}; X[H-k] mirrors it.
    float2* Xr = a.X + Xo;
    const float2* wp = a.tab + R * T + R * E;
    if (a.C == 1) {
        // w_{2H}^k for k = lt + per_trace j as w^{lt} w^{per_trace j}: one
        // coalesced table read per thread, then a broadcast one per pair
        const float2 w0 = __ldg(wp + lt);
        int kj = 0;
#pragma unroll 4
        for (int k = lt; k <= H / 2 && live; k += per_trace, kj += per_trace)
            unpack_pair(Xr, k, H, zs[pidx(k)], zs[pidx((H - k) & (H - 1))], cmul(w0, __ldg(wp + kj)));
    } else {
        const int P = (H >> 1) / a.C;
        const int k0 = rank * P;
        const int k1 = k0 + P + (rank == a.C - 1 ? 1 : 0);
        for (int k = k0 + lt; k < k1 && live; k += per_trace) {
            const float2 A = zs[pidx(k - k0)];
            const float2 B = (k == 0 || 2 * k == H) ? A : zs[pidx(P + 1 + (k - k0))];
            unpack_pair(Xr, k, H, A, B, __ldg(wp + k));
        }
    }
}

// Two-lane variant: each thread carries residues ra and ra + Rc/2 of one
// trace as the two packed lanes of a C2, so the packed input is read once per
// pair and the FFT arithmetic and twiddle loads are shared by both residues.
// Same staging and unpack as k_fft_real_padded.
template <int LZ>
__global__ void __launch_bounds__(256, 2) k_fft_real_padded2(FftArgs a) {
    using FFT = BlockFFT<LZ, false, C2>;
    constexpr int E = FFT::E;
    constexpr int T = FFT::T;
    extern __shared__ float4 smem4[];

    const int G = a.Rc >> 1;                     // residue pairs per CTA per trace
    const int per_trace = G * T;
    const int tid = threadIdx.x;
    const int f = tid / per_trace;
    const int lt = tid - f * per_trace;
    const int gl = lt / T;
    const int t = lt - gl * T;
    const int rank = a.C > 1 ? (int)(blockIdx.x % a.C) : 0;
    const int64_t b = (int64_t)(blockIdx.x / a.C) * a.F + f;
    const bool live = b < a.batch;
    int n = a.n;
    int64_t xo = (live ? b : 0) * a.ld_x, Xo = (live ? b : 0) * a.ld_X;
    if (a.items && live) {
        const RaggedItem& it = a.items[b];
        xo = it.x_off;
        Xo = it.out_off;
        n = it.n;
    }
    const int R = 1 << a.logR;
    const int ra = rank * a.Rc + gl;             // lane a residue
    const int rb = ra + G;                       // lane b residue
    const int H = a.H;
    float2* zs = reinterpret_cast<float2*>(smem4) + f * a.trace_smem;
    float4* s = reinterpret_cast<float4*>(zs) + gl * padded_len(LZ);

    C2 v[E];
    {
        // both lanes' pre-twiddles w_H^{r m} = w_H^{r t} w_H^{r T i} as one
        // packed product, then the shared z[m] times both
        const C2 wt = c2(__ldg(a.tab + ra * T + t), __ldg(a.tab + rb * T + t));
        const float2* wia = a.tab + R * T + ra * E;
        const float2* wib = a.tab + R * T + rb * E;
        const float* xr = a.x + xo;
        if (live && n >= 2 * LZ && (reinterpret_cast<uintptr_t>(xr) & 7) == 0) {
            // the trace covers every packed slot and the row is 8-byte
            // aligned: each packed sample z[m] is one 8-byte load
            const float2* x2 = reinterpret_cast<const float2*>(xr);
#pragma unroll
            for (int i = 0; i < E; ++i)
                v[i] = cmul(__ldg(x2 + t + T * i), cmul(wt, c2(__ldg(wia + i), __ldg(wib + i))));
        } else if (live && n >= 2 * LZ) {
            // full trace, odd row start: two 4-byte loads, no per-sample bounds
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int m = t + T * i;
                v[i] = cmul(make_float2(__ldg(xr + 2 * m), __ldg(xr + 2 * m + 1)),
                            cmul(wt, c2(__ldg(wia + i), __ldg(wib + i))));
            }
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int m = t + T * i;
                float re = 0.f, im = 0.f;
                if (live && 2 * m < n) re = __ldg(xr + 2 * m);
                if (live && 2 * m + 1 < n) im = __ldg(xr + 2 * m + 1);
                v[i] = cmul(make_float2(re, im), cmul(wt, c2(__ldg(wia + i), __ldg(wib + i))));
            }
        }
    }
    FFT::run(v, s, t, a.tw);

    // Every CTA of a cluster must have finished its FFT (whose exchanges use
    // this shared memory) before any of them writes Z into its peers.
    if (a.C > 1) cluster_arrive_relaxed_wait(); else __syncthreads();
    if (a.C == 1) {
        const int TR = T << a.logR;
        if ((TR & 15) == 0) {
            // Z[R (t + T i) + r] sits at pidx(R t + r) + 17 (T R/16) i
            const int st = (TR >> 4) * 17;
            float2* pa = zs + pidx((t << a.logR) + ra);
            float2* pb = zs + pidx((t << a.logR) + rb);
#pragma unroll
            for (int i = 0; i < E; ++i) {
                pa[st * i] = lane_a(v[i]);
                pb[st * i] = lane_b(v[i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int q = (t + T * i) << a.logR;
                zs[pidx(q + ra)] = lane_a(v[i]);
                zs[pidx(q + rb)] = lane_b(v[i]);
            }
        }
        __syncthreads();
    } else {
        cg::cluster_group cl = cg::this_cluster();
        const int logP = a.logChunk - 1;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int q = (t + T * i) << a.logR;
            const int2 ha = pair_home(q + ra, H, logP, a.C);
            const int2 hb = pair_home(q + rb, H, logP, a.C);
            dsmem_store(zs, pidx(ha.y), (unsigned)ha.x, lane_a(v[i]));
            dsmem_store(zs, pidx(hb.y), (unsigned)hb.x, lane_b(v[i]));
        }
        cl.sync();
    }

    float2* Xr = a.X + Xo;
    const float2* wp = a.tab + R * T + R * E;
    if (a.C == 1) {
        // w_{2H}^k for k = lt + per_trace j as w^{lt} w^{per_trace j}: one
        // coalesced table read per thread, then a broadcast one per pair
        const float2 w0 = __ldg(wp + lt);
        if ((per_trace & 15) == 0) {
            // Here H/2 = E per_trace, so k = lt + per_trace j (j < E) covers
            // [0, H/2) and thread 0 adds k = H/2.  With per_trace a multiple
            // of 16, pidx(k) and pidx(H - k) move by a constant step, so the
            // fully unrolled loop addresses everything from three bases.
            const int step = per_trace + (per_trace >> 4);
            const float2* za = zs + pidx(lt);
            const float2* zb = zs + pidx(H - lt);        // lt = 0: slot H/16 + H, not read at j = 0
            if (live) {
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const float2 A = za[step * j];
                    const float2 B = (j == 0 && lt == 0) ? A : zb[-step * j];
                    unpack_pair(Xr, lt + per_trace * j, H, A, B, cmul(w0, __ldg(wp + per_trace * j)));
                }
                if (lt == 0) {
                    const float2 Z = zs[pidx(H / 2)];
                    unpack_pair(Xr, H / 2, H, Z, Z, __ldg(wp + H / 2));
                }
            }
        } else {
            int kj = 0;
#pragma unroll 4
            for (int k = lt; k <= H / 2 && live; k += per_trace, kj += per_trace)
                unpack_pair(Xr, k, H, zs[pidx(k)], zs[pidx((H - k) & (H - 1))], cmul(w0, __ldg(wp + kj)));
        }
    } else {
        const int P = (H >> 1) / a.C;
        const int k0 = rank * P;
        const int k1 = k0 + P + (rank == a.C - 1 ? 1 : 0);
        for (int k = k0 + lt; k < k1 && live; k += per_trace) {
            const float2 A = zs[pidx(k - k0)];
            const float2 B = (k == 0 || 2 * k == H) ? A : zs[pidx(P + 1 + (k - k0))];
            unpack_pair(Xr, k, H, A, B, __ldg(wp + k));
        }
    }
}

// ---------------------------------------------------------------------------
// Two-lane kernel compiled for one (LZ, R) with one CTA per group of traces
// (C == 1): lanes a and b carry residues g and g + R/2 of one trace, as in
// k_fft_real_padded2, but every trace size, step and offset is a
// compile-time constant, and the tables are stored in the packed pair
// layout the two-lane arithmetic reads without register shuffles:
//   pre4[g][m] = (wa.x, wb.x, wa.y, wb.y), wa = w_H^{g m}, wb = w_H^{(g+R/2) m}
//   tw4[e]     = (c, c, s, s) for the BlockFFT<LZ> twiddle c + j s.
// Table layout after the generic part (fixed_table_offsets): see below.
__host__ __device__ constexpr int fixed_generic_entries(int LZ, int R) {
    return R * (LZ / 16) + R * 16 + R * LZ / 2 + 1;
}
// float4 index of pre4 and of tw4 in a table that starts 16-byte aligned
__host__ __device__ constexpr int fixed_pre4_index(int LZ, int R) { return (fixed_generic_entries(LZ, R) + 1) / 2; }
__host__ __device__ constexpr int fixed_tw4_index(int LZ, int R) { return fixed_pre4_index(LZ, R) + (R / 2) * LZ; }

// z (a packed sample pair) times the two lanes' pre-twiddles
__device__ __forceinline__ C2 pretwiddle2(float2 z, float4 w) {
    const float2 zx = make_float2(z.x, z.x), zy = make_float2(z.y, z.y);
    const float2 wr = make_float2(w.x, w.y), wi = make_float2(w.z, w.w);
    return C2{sub2(mul2(zx, wr), mul2(zy, wi)), fma2(zx, wi, mul2(zy, wr))};
}
// Folded input of two residues (lanes a, b): (z0 + z1 c_lane) w_lane, with
// c = (ca.x, cb.x, ca.y, cb.y) and w packed the same way
__device__ __forceinline__ C2 pretwiddle2_fold(float2 z0, float2 z1, float4 c, float4 w) {
    const float2 cr = make_float2(c.x, c.y), ci = make_float2(c.z, c.w);
    const float2 z1x = make_float2(z1.x, z1.x), z1y = make_float2(z1.y, z1.y);
    const float2 zx = fma2(z1x, cr, fma2(make_float2(-z1.y, -z1.y), ci, make_float2(z0.x, z0.x)));
    const float2 zy = fma2(z1x, ci, fma2(z1y, cr, make_float2(z0.y, z0.y)));
    const float2 wr = make_float2(w.x, w.y), wi = make_float2(w.z, w.w);
    return C2{sub2(mul2(zx, wr), mul2(zy, wi)), fma2(zx, wi, mul2(zy, wr))};
}

// X[k], X[H - k] from A = Z[k], B = Z[H - k], w = e^{-j pi k/H}/2 (the 1/2
// of the real-input unpack folded into w), 0 < k < H/2
template <int H>
__device__ __forceinline__ void unpack_pair_half(float2* Xr, int k, float2 A, float2 B, float2 w) {
    const float sx = A.x + B.x, sy = A.y - B.y;
    const float dx = A.x - B.x, dy = A.y + B.y;
    const float p = fmaf(w.x, dx, -w.y * dy), q = fmaf(w.x, dy, w.y * dx);   // w (A - conj B)
    Xr[k] = make_float2(fmaf(0.5f, sx, q), fmaf(0.5f, sy, -p));
    Xr[H - k] = make_float2(fmaf(0.5f, sx, -q), fmaf(-0.5f, sy, -p));
}

template <int LZ, int R>
__global__ void __launch_bounds__(256, 2) k_fft_real_padded2r(FftArgs a) {
    constexpr int T = LZ / 16, E = 16, G = R / 2, PT = G * T;
    constexpr int F = PT >= 256 ? 1 : 256 / PT;
    constexpr int H = R * LZ;
    constexpr int TS = padded_len(H) + 2;          // float2 per trace (even: float4 views)
    using FFT = BlockFFT<LZ, false, C2, 16, float4>;
    static_assert(PT * E == H / 2, "one CTA holds the trace's residue pairs");
    extern __shared__ float4 smem4[];

    const int tid = threadIdx.x;
    const int f = tid / PT;
    const int lt = tid - f * PT;
    const int gl = lt / T;
    const int t = lt - gl * T;
    const int64_t b = (int64_t)blockIdx.x * F + f;
    const bool live = b < a.batch;
    int n = a.n;
    int64_t xo = (live ? b : 0) * a.ld_x, Xo = (live ? b : 0) * a.ld_X;
    if (a.items && live) {
        const RaggedItem& it = a.items[b];
        xo = it.x_off;
        Xo = it.out_off;
        n = it.n;
    }
    float2* zs = reinterpret_cast<float2*>(smem4) + f * TS;
    float4* s = reinterpret_cast<float4*>(zs) + gl * padded_len(LZ);
    const float4* tab4 = reinterpret_cast<const float4*>(a.tab);

    C2 v[E];
    {
        const float4* w4 = tab4 + fixed_pre4_index(LZ, R) + gl * LZ + t;
        const float* xr = a.x + xo;
        if (live && n >= 2 * LZ && (reinterpret_cast<uintptr_t>(xr) & 7) == 0) {
            const float2* x2 = reinterpret_cast<const float2*>(xr) + t;
#pragma unroll
            for (int i = 0; i < E; ++i) v[i] = pretwiddle2(__ldg(x2 + T * i), __ldg(w4 + T * i));
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int m = t + T * i;
                float re = 0.f, im = 0.f;
                if (live && 2 * m < n) re = __ldg(xr + 2 * m);
                if (live && 2 * m + 1 < n) im = __ldg(xr + 2 * m + 1);
                v[i] = pretwiddle2(make_float2(re, im), __ldg(w4 + T * i));
            }
        }
    }
    FFT::run(v, s, t, tab4 + fixed_tw4_index(LZ, R));

    // Z[R q + r] for the lanes' residues, q = t + T i, in natural order
    __syncthreads();
    {
        constexpr int ST = 17 * (T * R / 16);      // pidx step of q -> q + T
        static_assert((T * R) % 16 == 0, "constant staging step");
        float2* pa = zs + pidx(t * R + gl);
        float2* pb = zs + pidx(t * R + gl + G);
#pragma unroll
        for (int i = 0; i < E; ++i) {
            pa[ST * i] = lane_a(v[i]);
            pb[ST * i] = lane_b(v[i]);
        }
    }
    __syncthreads();
    if (!live) return;

    // unpack the pairs (k, H - k), k = lt + PT j (j < E) covering [0, H/2),
    // plus k = H/2; the twiddle w_{2H}^k/2 = (w^{lt}/2) w^{PT j}
    float2* Xr = a.X + Xo;
    const float2* wp = a.tab + R * T + R * E;
    const float2 w0 = cscale(__ldg(wp + lt), 0.5f);
    constexpr int STEP = PT + PT / 16;
    static_assert(PT % 16 == 0, "constant unpack step");
    const float2* za = zs + pidx(lt);
    const float2* zb = zs + pidx(H - lt);
    if (lt == 0) {
        // k = 0: X[0] = Re Z0 + Im Z0, X[H] = Re Z0 - Im Z0; k = H/2: conj
        const float2 Z0 = zs[0];
        Xr[0] = make_float2(Z0.x + Z0.y, 0.f);
        Xr[H] = make_float2(Z0.x - Z0.y, 0.f);
        const float2 Zh = zs[pidx(H / 2)];
        Xr[H / 2] = make_float2(Zh.x, -Zh.y);
    } else {
        unpack_pair_half<H>(Xr, lt, za[0], zb[0], w0);
    }
#pragma unroll
    for (int j = 1; j < E; ++j)
        unpack_pair_half<H>(Xr, lt + PT * j, za[STEP * j], zb[-STEP * j], cmul(w0, __ldg(wp + PT * j)));
}

// ---------------------------------------------------------------------------
// Two-lane kernel with the last Stockham pass fused into the unpack, for
// (LZ, R) whose BlockFFT<LZ> has three passes (radix 16, 16, rho; LZ = 512
// has rho = 2, LZ = 1024 rho = 4).  The kernels above run all three passes,
// store Z to shared memory and read it back for the unpack; here the outputs
// of the second pass go straight to the staging area, and each unpack thread
// computes the rho-point butterflies whose outputs it needs:
//
//   Z[k + n H/rho] (n < rho) are the outputs of butterfly j = k/R of residue
//   r = k mod R, and their mirrors Z[H - k - n H/rho] are the outputs of one
//   butterfly of residue R - r (of residue 0 for r = 0), whose inputs sit at
//   staging slots (m + 1) H/rho - k.  So one thread reads 2 rho values,
//   computes two butterflies and forms the 2 rho outputs X[k + n H/rho] and
//   X[H - k - n H/rho] (k < H/(2 rho)), every Z value read once.
//
// That removes one shared-memory exchange of the whole trace and the third
// pass's twiddle loads, which matters because the two-lane kernels are bound
// by the L1 / shared-memory data pipe (ncu: lsu wavefronts at 84% of peak),
// not by DRAM.  Lanes a and b carry residues 2p and 2p + 1, so the staged
// pair is one 16-byte store; the staging slot of x = pos R + r (float2 units)
// XORs the 16-byte chunk index within each 128-byte row with the row index
// (mod 8), which keeps the stride-R stores and the consecutive-k reads free
// of bank conflicts without padding.
//
// Table (float4 units): pre4 [R/2][LZ] = (wa.x, wb.x, wa.y, wb.y),
// wa = w_H^{2p m}, wb = w_H^{(2p+1) m}; ub4 [PT] = (w_{2H}^{lt}/2,
// w_LZ^{lt/R}); then (float2 units) um [PT] = w_LZ^{j'(lt)}, the mirror
// butterfly index of k = lt, and the BlockFFT<LZ> twiddles as (c, s) (8 bytes
// a twiddle: the float4 (c, c, s, s) form measured 2% slower, the extra L1
// traffic costing more than the register moves it saves).  The per-k
// twiddles are ub4 and um times compile-time constants (k = lt + PT j:
// w_{2H}^{PT j} = e^{-j pi j/32}, w_LZ^{(PT/R) j} = e^{-j 2 pi j/32}).
//
// Folded form (FOLD = 2): traces of up to 2 LZ sample pairs with R = H/LZ
// residues of LZ points, z[m0] and z[m0 + LZ] summed before the residue FFT:
//   Z[R q + r] = sum_{m0 < LZ} w_H^{m0 r} (z[m0] + z[m0 + LZ] w_R^r) w_LZ^{m0 q}
// (w_H^{LZ r} = w_R^r, w_H^{LZ R q} = 1).  This lets a trace of 2 LZ pairs
// use the kernel of LZ-point residues (LZ = 512: radix 16, 16, 2, each pair
// of residues one warp) instead of 2 LZ-point ones.  The table then holds,
// after pre4, fold4 [R/2] = (w_R^{2p}, w_R^{2p+1}) packed like pre4.
__host__ __device__ constexpr int fused_fold4_index(int LZ, int R) { return (R / 2) * LZ; }
__host__ __device__ constexpr int fused_ub4_index(int LZ, int R, int FOLD = 1) {
    return (R / 2) * LZ + (FOLD > 1 ? R / 2 : 0);
}
__host__ __device__ constexpr int fused_um_index(int LZ, int R, int FOLD = 1) {
    return 2 * (fused_ub4_index(LZ, R, FOLD) + (R / 2) * (LZ / 16));
}
__host__ __device__ constexpr int fused_tw2_index(int LZ, int R, int FOLD = 1) {
    return fused_um_index(LZ, R, FOLD) + (R / 2) * (LZ / 16);
}
__host__ __device__ constexpr int fused_entries(int LZ, int R, int FOLD = 1) {
    return fused_tw2_index(LZ, R, FOLD) + fft_twiddle_entries(LZ);
}
// float2 per trace: the BlockFFT exchange areas of the R/2 pairs (the staged
// H values fit in the same space)
__host__ __device__ constexpr int fused_trace_smem(int LZ, int R) { return (R / 2) * padded_len(LZ) * 2; }

// staging slot of x (float2 units)
__device__ __forceinline__ int fsw(int x) { return x ^ (((x >> 4) & 7) << 1); }

// b_m = y_m w^m, then the rho-point DFT in place (natural output order)
template <int RHO>
__device__ __forceinline__ void fused_butterfly(float2 (&y)[RHO], float2 w) {
    if constexpr (RHO == 2) {
        y[1] = cmul(y[1], w);
        dft2<false>(y[0], y[1]);
    } else {
        const float2 w2 = cmul(w, w);
        const float2 w3 = cmul(w2, w);
        y[1] = cmul(y[1], w);
        y[2] = cmul(y[2], w2);
        y[3] = cmul(y[3], w3);
        dft4<false>(y[0], y[1], y[2], y[3]);
    }
}

// Passes 0 and 1 of the residue pair's BlockFFT on v (pre-twiddled input
// m = t + (LZ/16) i), the staging of their outputs and the fused third pass
// with the unpack into Xr.  Every thread of the CTA calls it (it holds
// __syncthreads); threads of a trace slot without a trace pass live = false.
// (bar, nthr): the trace's barrier (group_sync); pbar: the barrier of the
// residue pair's exchange (-1: the pair is one warp), 64 threads.
template <int LZ, int R, int FOLD = 1>
__device__ __forceinline__ void fused_fft_unpack(C2 (&v)[16], float2* zs, int gl, int t, int lt, bool live,
                                                 float2* Xr, const float2* tab, int bar, int nthr, int pbar) {
    using S = FFTShape<LZ, 16>;
    static_assert(S::NPASS == 3 && S::NPB == 2, "fused kernel: radix 16, 16, rho");
    constexpr int RHO = S::REM;
    static_assert(RHO == 2 || RHO == 4, "fused butterflies of radix 2 or 4");
    constexpr int T = LZ / 16, G = R / 2, PT = G * T;
    constexpr int H = R * LZ;
    constexpr int HB = H / RHO;          // outputs k + n HB share a butterfly
    constexpr int J = 16 / RHO;          // k values per thread
    static_assert(PT * J * 2 * RHO == H, "every output once");
    static_assert(PT % 128 == 0 && HB % 128 == 0, "staging swizzle constant along j and m");
    static_assert(PT / R * 32 == LZ, "q steps by LZ/32 along j");
    const float4* tab4 = reinterpret_cast<const float4*>(tab);
    using FFT = BlockFFT<LZ, false, C2, 16, float2>;
    // the exchange between passes 0 and 1 touches only the pair's own area
    FFT::template run_first<2>(v, reinterpret_cast<float4*>(zs) + gl * padded_len(LZ), t,
                               tab + fused_tw2_index(LZ, R, FOLD), pbar, T);

    // outputs of pass 1 (radix 16, span 16): v[r] is position base + 16 r of
    // residues 2 gl and 2 gl + 1, staged at x = pos R + 2 gl
    group_sync(bar, nthr);
    {
        const int k16 = t & 15;
        const int pos0 = (t - k16) * 16 + k16;
        float4* st4 = reinterpret_cast<float4*>(zs);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int x = (pos0 + 16 * r) * R + 2 * gl;
            st4[fsw(x) >> 1] = make_float4(v[r].re.x, v[r].im.x, v[r].re.y, v[r].im.y);
        }
    }
    group_sync(bar, nthr);
    if (!live) return;

    const float4 ub = __ldg(tab4 + fused_ub4_index(LZ, R, FOLD) + lt);
    const float2 wk0 = make_float2(ub.x, ub.y);    // w_{2H}^{lt} / 2
    const float2 wq0 = make_float2(ub.z, ub.w);    // w_LZ^{lt/R}
    const float2 wm0 = __ldg(tab + fused_um_index(LZ, R, FOLD) + lt);
    // the swizzle depends only on the low 7 bits of x, and PT j, m HB are
    // multiples of 128: every slot below is a base plus a constant
    const float2* zf = zs + fsw(lt);
    const float2* zm = zs + fsw(HB - lt) - HB;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        if (j == 0 && lt == 0) continue;           // k = 0: below
        const float2 wq = cmul(wq0, wpi32(2 * j));   // w_LZ^{q}, q = k/R
        const float2 wm = cmulc(wm0, wpi32(2 * j));  // w_LZ^{j'}, the mirror butterfly
        const float2 wk = cmul(wk0, wpi32(j));        // w_{2H}^k / 2
        float2 A[RHO], B[RHO];
#pragma unroll
        for (int m = 0; m < RHO; ++m) {
            A[m] = zf[PT * j + m * HB];
            B[m] = zm[(m + 1) * HB - PT * j];
        }
        fused_butterfly<RHO>(A, wq);               // A[n] = Z[k + n HB]
        fused_butterfly<RHO>(B, wm);               // B[n] = Z[(n + 1) HB - k]
        // pairs (k + n HB, H - k - n HB), twiddle w_{2H}^{k + n HB}/2
        const int k = lt + PT * j;
        unpack_pair_half<H>(Xr, k, A[0], B[RHO - 1], wk);
        unpack_pair_half<H>(Xr, k + HB, A[1], B[RHO - 2], rot_pi32<32 / RHO>(wk));
        if constexpr (RHO == 4) {
            unpack_pair_half<H>(Xr, k + 2 * HB, A[2], B[1], rot_pi32<16>(wk));
            unpack_pair_half<H>(Xr, k + 3 * HB, A[3], B[0], rot_pi32<24>(wk));
        }
    }
    if (lt == 0) {
        // k = 0: butterfly 0 of residue 0 (no twiddles): Z[n HB]
        float2 A[RHO];
#pragma unroll
        for (int m = 0; m < RHO; ++m) A[m] = zs[fsw(m * HB)];
        fused_butterfly<RHO>(A, make_float2(1.f, 0.f));
        Xr[0] = make_float2(A[0].x + A[0].y, 0.f);
        Xr[H] = make_float2(A[0].x - A[0].y, 0.f);
        if constexpr (RHO == 4) unpack_pair_half<H>(Xr, HB, A[1], A[3], make_float2(0.5f * kS2, -0.5f * kS2));
        Xr[H / 2] = make_float2(A[RHO / 2].x, -A[RHO / 2].y);
        // k = HB/2: butterfly NS/2 of residue 0, twiddle w_LZ^{NS/2} = e^{-j pi/rho}
#pragma unroll
        for (int m = 0; m < RHO; ++m) A[m] = zs[fsw(HB / 2 + m * HB)];
        fused_butterfly<RHO>(A, wpi32(32 / RHO));
        // pairs (HB/2 + n HB, H - HB/2 - n HB), twiddle e^{-j pi (2n+1)/(2 rho)}/2
        unpack_pair_half<H>(Xr, HB / 2, A[0], A[RHO - 1], cscale(wpi32(16 / RHO), 0.5f));
        if constexpr (RHO == 4) unpack_pair_half<H>(Xr, HB / 2 + HB, A[1], A[2], cscale(wpi32(48 / RHO), 0.5f));
    }
}

template <int LZ, int R, int FOLD = 1>
__global__ void __launch_bounds__(256, 2) k_fft_real_fused(FftArgs a) {
    constexpr int T = LZ / 16, E = 16, G = R / 2, PT = G * T;
    constexpr int F = PT >= 256 ? 1 : 256 / PT;
    constexpr int TS = fused_trace_smem(LZ, R);
    extern __shared__ float4 smem4[];

    const int tid = threadIdx.x;
    const int f = tid / PT;
    const int lt = tid - f * PT;
    const int gl = lt / T;
    const int t = lt - gl * T;
    const int64_t b = (int64_t)blockIdx.x * F + f;
    const bool live = b < a.batch;
    int n = a.n;
    int64_t xo = (live ? b : 0) * a.ld_x, Xo = (live ? b : 0) * a.ld_X;
    if (a.items && live) {
        const RaggedItem& it = a.items[b];
        xo = it.x_off;
        Xo = it.out_off;
        n = it.n;
    }
    const float4* w4 = reinterpret_cast<const float4*>(a.tab) + gl * LZ + t;
    C2 v[E];
    const float* xr = a.x + xo;
    if constexpr (FOLD == 1) {
        if (live && n >= 2 * LZ && (reinterpret_cast<uintptr_t>(xr) & 7) == 0) {
            const float2* x2 = reinterpret_cast<const float2*>(xr) + t;
#pragma unroll
            for (int i = 0; i < E; ++i) v[i] = pretwiddle2(__ldg(x2 + T * i), __ldg(w4 + T * i));
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int m = t + T * i;
                float re = 0.f, im = 0.f;
                if (live && 2 * m < n) re = __ldg(xr + 2 * m);
                if (live && 2 * m + 1 < n) im = __ldg(xr + 2 * m + 1);
                v[i] = pretwiddle2(make_float2(re, im), __ldg(w4 + T * i));
            }
        }
    } else {
        static_assert(FOLD == 2, "fold of two");
        const float4 c4 = __ldg(reinterpret_cast<const float4*>(a.tab) + fused_fold4_index(LZ, R) + gl);
        if (live && n >= 4 * LZ && (reinterpret_cast<uintptr_t>(xr) & 7) == 0) {
            const float2* x2 = reinterpret_cast<const float2*>(xr) + t;
#pragma unroll
            for (int i = 0; i < E; ++i)
                v[i] = pretwiddle2_fold(__ldg(x2 + T * i), __ldg(x2 + LZ + T * i), c4, __ldg(w4 + T * i));
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int m = t + T * i, m1 = m + LZ;
                float2 z0 = make_float2(0.f, 0.f), z1 = make_float2(0.f, 0.f);
                if (live && 2 * m < n) z0.x = __ldg(xr + 2 * m);
                if (live && 2 * m + 1 < n) z0.y = __ldg(xr + 2 * m + 1);
                if (live && 2 * m1 < n) z1.x = __ldg(xr + 2 * m1);
                if (live && 2 * m1 + 1 < n) z1.y = __ldg(xr + 2 * m1 + 1);
                v[i] = pretwiddle2_fold(z0, z1, c4, __ldg(w4 + T * i));
            }
        }
    }
    // F > 1: each trace's threads synchronise on their own named barrier;
    // each residue pair's exchange on its warp (T = 32) or on a named
    // barrier of its two warps (ids after the traces')
    static_assert(T == 32 || (T == 64 && F + F * G < 8), "barrier ids");
    fused_fft_unpack<LZ, R, FOLD>(v, reinterpret_cast<float2*>(smem4) + f * TS, gl, t, lt, live, a.X + Xo,
                                  a.tab, F > 1 ? 1 + f : 0, PT, T == 32 ? -1 : 1 + F + f * G + gl);
}

// Persistent form for whole rows at 16-byte aligned addresses (n = 2 LZ,
// 16-byte row pitch, no ragged items): two CTAs per SM loop over groups of F
// traces, and while a group is transformed one thread has the next group's
// rows copied into shared memory by the bulk-copy engine (cp.async.bulk,
// completion counted on an mbarrier per buffer), so that no warp waits on
// HBM latency for its input.  Every wait is bounded: one that gives up sets
// the context's status word, and the CTA leaves at the next group boundary
// after waiting (bounded) for the copies it still has in flight.
__host__ __device__ constexpr size_t fused_tma_smem(int LZ, int R) {
    return ((size_t)(256 / ((R / 2) * (LZ / 16)) > 1 ? 256 / ((R / 2) * (LZ / 16)) : 1)) *
               ((size_t)fused_trace_smem(LZ, R) * sizeof(float2) + 2 * (size_t)(2 * LZ) * sizeof(float)) + 16;
}

template <int LZ, int R>
__global__ void __launch_bounds__(256, 2) k_fft_real_fused_tma(FftArgs a) {
    constexpr int T = LZ / 16, E = 16, G = R / 2, PT = G * T;
    constexpr int F = PT >= 256 ? 1 : 256 / PT;
    constexpr int TS = fused_trace_smem(LZ, R);
    constexpr int XB = 2 * LZ;                       // floats of one row
    extern __shared__ float4 smem4[];
    float2* zs_all = reinterpret_cast<float2*>(smem4);
    float* xbuf = reinterpret_cast<float*>(zs_all + F * TS);        // [2][F][XB]
    uint64_t* bars = reinterpret_cast<uint64_t*>(xbuf + 2 * F * XB);
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int f = tid / PT;
    const int lt = tid - f * PT;
    const int gl = lt / T;
    const int t = lt - gl * T;
    const int64_t groups = (a.batch + F - 1) / F;
    const Guard guard{&abort_flag, a.status, a.timeout_ns};
    if (tid == 0) {
        abort_flag = 0;
        mbar_init(bars, 1);
        mbar_init(bars + 1, 1);
        mbar_init_fence();
    }
    __syncthreads();
    // thread 0: copies issued per buffer (the parity of a use is its count mod 2)
    uint32_t issued0 = 0, issued1 = 0;
    auto issue = [&](int64_t g, int buf) {
        const int nl = (int)(a.batch - g * F < F ? a.batch - g * F : F);
        mbar_expect_tx(bars + buf, (uint32_t)(nl * XB * sizeof(float)));
        for (int q = 0; q < nl; ++q)
            bulk_load(xbuf + (buf * F + q) * XB, a.x + (g * F + q) * a.ld_x, (uint32_t)(XB * sizeof(float)), bars + buf);
        if (buf) ++issued1;
        else ++issued0;
    };
    int64_t g = blockIdx.x;
    if (tid == 0 && g < groups) issue(g, 0);
    const float4* w4 = reinterpret_cast<const float4*>(a.tab) + gl * LZ + t;
    for (int it = 0; g < groups; ++it, g += gridDim.x) {
        const int buf = it & 1;
        __syncthreads();            // the last group's reads of zs and of xbuf[buf ^ 1] are done
        if (abort_flag) break;
        if (tid == 0 && g + gridDim.x < groups) issue(g + gridDim.x, buf ^ 1);
        wait_bounded(bars + buf, (uint32_t)((it >> 1) & 1), guard);
        const int64_t b = g * F + f;
        const bool live = b < a.batch;
        const float2* x2 = reinterpret_cast<const float2*>(xbuf + (buf * F + f) * XB) + t;
        C2 v[E];
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = pretwiddle2(live ? x2[T * i] : make_float2(0.f, 0.f), __ldg(w4 + T * i));
        fused_fft_unpack<LZ, R>(v, zs_all + f * TS, gl, t, lt, live, a.X + (live ? b : 0) * a.ld_X, a.tab, 0, 0, 0);
    }
    // after an abort: no copy may still be writing into this CTA's memory
    if (tid == 0 && abort_flag) {
        for (int q = 0; q < 2; ++q) {
            const uint32_t n_is = q ? issued1 : issued0;
            if (n_is == 0) continue;
            const uint64_t t0 = gtime();
            while (!mbar_try_wait(bars + q, (n_is - 1) & 1) && gtime() - t0 < a.timeout_ns) {
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Traces too long for one CTA (R/2 residue pairs of LZ/16 threads exceed 256
// threads): a thread-block cluster of C CTAs per trace, each CTA computing
// 256/(LZ/16) residue pairs, and the spectrum assembled in the CTAs' shared
// memory so that every HBM store is a contiguous run.
//
// Pair g >= 1 holds residues g and R - g.  Lane a transforms z[m] w_H^{g m};
// lane b transforms conj(z[m]) w_H^{g m}, whose LZ-point FFT at q is
// conj(Z[H - (R q + g)]) (the DFT of a conjugated sequence is the conjugated,
// index-reversed DFT, and w_H^{R m} = w_LZ^m shifts that reversal to
// LZ - 1 - q).  So after the FFT each thread holds, at every q, both members
// A = Z[k], B' = conj Z[H - k] of its unpack pairs (k, H - k), k = R q + g,
// and forms X[k] and X[H - k] in registers.  Pair 0 holds residues 0 and
// R/2, each its own mirror (Z[R q] pairs with Z[R (LZ - q)], Z[R q + R/2]
// with Z[R (LZ - 1 - q) + R/2]); it exchanges through its own shared memory
// and forms X[R q] and X[R q + R/2].
//
// CTA c of the cluster owns X[8192 c .. 8192 c + 8191] (the last one also
// X[H]): every output is stored once into its owner's shared memory
// (distributed shared memory; padded index o + o/8, which keeps the stride-R
// stores of a warp on distinct banks), and after a cluster barrier each CTA
// writes its run to HBM with coalesced stores.
//
// Table (float2 units): [H/2 + 1: w_{2H}^k] [pad] [pre: R/2 rows of LZ:
// row 0 w_H^{(R/2) m}, row g w_H^{g m}] [BlockFFT<LZ> twiddles (c, c, s, s)].
constexpr int kClusterRun = 8192;          // outputs owned by one CTA
__host__ __device__ constexpr int pidx8(int o) { return o + (o >> 3); }
__host__ __device__ constexpr int cluster_pre_offset(int H) { return ((H / 2 + 1) + 1) & ~1; }
__host__ __device__ constexpr int cluster_tw4_index(int H) { return (cluster_pre_offset(H) + H / 2) / 2; }

// X[k] from A = Z[k] and Bc = conj Z[H - k], wh = e^{-j pi k/H}/2
__device__ __forceinline__ float2 unpack_fwd(float2 A, float2 Bc, float2 wh) {
    const float sx = A.x + Bc.x, sy = A.y + Bc.y;     // A + conj B
    const float dx = A.x - Bc.x, dy = A.y - Bc.y;     // A - conj B
    const float p = fmaf(wh.x, dx, -wh.y * dy), q = fmaf(wh.x, dy, wh.y * dx);
    return make_float2(fmaf(0.5f, sx, q), fmaf(0.5f, sy, -p));
}
// X[H - k] from the same A, Bc and wh (conj of the mirrored formula)
__device__ __forceinline__ float2 unpack_mirror(float2 A, float2 Bc, float2 wh) {
    const float sx = A.x + Bc.x, sy = A.y + Bc.y;
    const float dx = A.x - Bc.x, dy = A.y - Bc.y;
    const float p = fmaf(wh.x, dx, -wh.y * dy), q = fmaf(wh.x, dy, wh.y * dx);
    return make_float2(fmaf(0.5f, sx, -q), fmaf(-0.5f, sy, -p));
}

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

template <int LZ, int R>
__global__ void __launch_bounds__(256, 2) k_fft_real_cluster(FftArgs a) {
    constexpr int T = LZ / 16, E = 16, PPC = 256 / T, NP = R / 2, C = NP / PPC;
    constexpr int H = R * LZ;
    static_assert(C >= 2 && C <= 8, "a portable cluster");
    static_assert(H / C == kClusterRun, "each CTA owns 8192 outputs");
    using FFT = BlockFFT<LZ, false, C2, 16, float4>;
    extern __shared__ float4 smem4[];

    const int tid = threadIdx.x;
    const int gl = tid / T;
    const int t = tid - gl * T;
    const int c = (int)cluster_rank();
    const int g = c * PPC + gl;                      // residue pair of this thread group
    const int64_t b = (int64_t)(blockIdx.x / C);     // one trace per cluster
    const bool live = b < a.batch;
    int n = a.n;
    int64_t xo = (live ? b : 0) * a.ld_x, Xo = (live ? b : 0) * a.ld_X;
    if (a.items && live) {
        const RaggedItem& it = a.items[b];
        xo = it.x_off;
        Xo = it.out_off;
        n = it.n;
    }
    float4* s = smem4 + gl * padded_len(LZ);
    const float2* wk = a.tab;                                     // w_{2H}^k, k <= H/2
    const float2* pre = a.tab + cluster_pre_offset(H) + g * LZ;
    const float4* tw4 = reinterpret_cast<const float4*>(a.tab) + cluster_tw4_index(H);

    // 1. packed, pre-twiddled input (lane b conjugated for pairs g >= 1)
    C2 v[E];
    {
        const float* xr = a.x + xo;
        const bool full = live && n >= 2 * LZ && (reinterpret_cast<uintptr_t>(xr) & 7) == 0;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int m = t + T * i;
            float2 z;
            if (full) {
                z = __ldg(reinterpret_cast<const float2*>(xr) + m);
            } else {
                z.x = (live && 2 * m < n) ? __ldg(xr + 2 * m) : 0.f;
                z.y = (live && 2 * m + 1 < n) ? __ldg(xr + 2 * m + 1) : 0.f;
            }
            const float2 w = __ldg(pre + m);
            if (g != 0) {
                const float P = z.x * w.x, Q = z.y * w.y, S = z.x * w.y, U = z.y * w.x;
                v[i] = C2{make_float2(P - Q, P + Q), make_float2(S + U, S - U)};
            } else {
                v[i] = C2{make_float2(z.x, fmaf(z.x, w.x, -z.y * w.y)), make_float2(z.y, fmaf(z.x, w.y, z.y * w.x))};
            }
        }
    }
    FFT::run(v, s, t, tw4);

    // 2. pair 0: stage Z[R q] and Z[R q + R/2] (natural order in q)
    __syncthreads();
    float2* z0 = reinterpret_cast<float2*>(s);
    float2* z4 = z0 + padded_len(LZ);
    if (g == 0) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            z0[pidx(t + T * i)] = lane_a(v[i]);
            z4[pidx(t + T * i)] = lane_b(v[i]);
        }
    }
    __syncthreads();

    // 3. outputs in registers: out[2 i] at k0_i, out[2 i + 1] at k1_i
    float2 out[2 * E];
    const float2 wb0 = cscale(__ldg(wk + R * t + g), 0.5f);
    const float2 wb4 = cscale(__ldg(wk + R * t + R / 2), 0.5f);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const float ci = i <= 8 ? cos_pi16(i) : -cos_pi16(16 - i);
        const float si = i <= 8 ? cos_pi16(8 - i) : cos_pi16(i - 8);
        const float2 ei = make_float2(ci, -si);                  // e^{-j pi i/16}
        const int q = t + T * i;
        if (g != 0) {
            const float2 wh = cmul(wb0, ei);
            out[2 * i] = unpack_fwd(lane_a(v[i]), lane_b(v[i]), wh);
            out[2 * i + 1] = unpack_mirror(lane_a(v[i]), lane_b(v[i]), wh);
        } else {
            const float2 A0 = lane_a(v[i]), B0 = z0[pidx((LZ - q) & (LZ - 1))];
            const float2 A4 = lane_b(v[i]), B4 = z4[pidx(LZ - 1 - q)];
            out[2 * i] = unpack_fwd(A0, make_float2(B0.x, -B0.y), cmul(wb0, ei));
            out[2 * i + 1] = unpack_fwd(A4, make_float2(B4.x, -B4.y), cmul(wb4, ei));
        }
    }
    float2 xh = make_float2(0.f, 0.f);                            // X[H] (pair 0, q = 0)
    if (g == 0 && t == 0) {
        const float2 Z0 = lane_a(v[0]);
        xh = make_float2(Z0.x - Z0.y, 0.f);
    }

    // 4. every CTA of the cluster is done with its shared memory: store each
    //    output into its owner's run
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    float2* run = reinterpret_cast<float2*>(smem4);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int q = t + T * i;
        const int k0 = g != 0 ? R * q + g : R * q;
        const int k1 = g != 0 ? H - (R * q + g) : R * q + R / 2;
        dsmem_store(run, pidx8(k0 & (kClusterRun - 1)), (unsigned)(k0 / kClusterRun), out[2 * i]);
        dsmem_store(run, pidx8(k1 & (kClusterRun - 1)), (unsigned)(k1 / kClusterRun), out[2 * i + 1]);
    }
    if (g == 0 && t == 0) dsmem_store(run, pidx8(kClusterRun), (unsigned)(C - 1), xh);
    cl.sync();

    // 5. coalesced run to HBM
    if (!live) return;
    float2* Xr = a.X + Xo + (int64_t)c * kClusterRun;
#pragma unroll 4
    for (int o = tid; o < kClusterRun; o += 256) Xr[o] = run[pidx8(o)];
    if (c == C - 1 && tid == 0) Xr[kClusterRun] = run[pidx8(kClusterRun)];
}

// ---------------------------------------------------------------------------
// Ragged batches as one persistent launch (work queue).  Every trace has its
// own N and N_FFT; R = H/LZ residue FFTs of LZ <= 4096 points each.  A unit is
// the work of one 256-thread CTA (two per SM):
//   mode 0: F = 256/(R/2 LZ/16) whole traces, two residues per thread as
//           packed lanes (g, g + R/2), Z staged in natural order and unpacked
//           with coalesced stores (as k_fft_real_padded2);
//   mode 1: G = 256/(LZ/16) residue pairs of one trace that does not fit one
//           CTA.  Pair g >= 1 carries residues g and R - g: lane a transforms
//           z[m] w_H^{g m}, lane b conj(z[m]) w_H^{g m}, whose FFT at q is
//           conj Z[H - (R q + g)], so each thread forms X[R q + g] and
//           X[H - R q - g] in registers.  Pair 0 (residues 0 and R/2, each its
//           own mirror) exchanges through shared memory.
// Units are sorted on the host (largest first) and popped from an atomic
// counter by persistent CTAs, two per SM.
struct FftQueueArgs {
    const RaggedItem* items;
    const FftUnit* units;
    int nunits;
    unsigned* counter;
    const float* x;
    float2* X;
    const float2* btw;       // BlockFFT twiddles of every size (radix-16 layout)
    float2* ws;              // mode 2: per-CTA workspace of ws_per_cta complex values
    int64_t ws_per_cta;
};

constexpr int kFftQueueThreads = 256;     // two CTAs per SM at 128 registers

// mode 0: F whole traces per CTA (the two-lane kernel's C == 1 path)
template <int LZ>
__device__ __forceinline__ void fft_queue_full(const FftQueueArgs& a, const FftUnit& u, float4* smem4) {
    using FFT = BlockFFT<LZ, false, C2>;
    constexpr int E = FFT::E, T = FFT::T;
    const int R = 1 << u.logR;
    const int G = R >> 1;
    const int H = R * LZ;
    const int PT = G * T;                                      // threads per trace
    const int TS = padded_len(H) + 2;                          // float2 per trace
    const int tid = threadIdx.x;
    const int f = tid / PT;
    const int lt = tid - f * PT;
    const int gl = lt / T;
    const int t = lt - gl * T;
    const bool live = f < u.count;
    const RaggedItem it = a.items[u.item + (live ? f : 0)];
    const int n = it.n;
    float2* zs = reinterpret_cast<float2*>(smem4) + f * TS;
    float4* s = reinterpret_cast<float4*>(zs) + gl * padded_len(LZ);
    const float2* tab = u.tab;
    const int ra = gl, rb = gl + G;

    C2 v[E];
    {
        const C2 wt = c2(__ldg(tab + ra * T + t), __ldg(tab + rb * T + t));
        const float2* wia = tab + R * T + ra * E;
        const float2* wib = tab + R * T + rb * E;
        const float* xr = a.x + it.x_off;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int m = t + T * i;
            float re = 0.f, im = 0.f;
            if (live && 2 * m < n) re = __ldg(xr + 2 * m);
            if (live && 2 * m + 1 < n) im = __ldg(xr + 2 * m + 1);
            v[i] = cmul(make_float2(re, im), cmul(wt, c2(__ldg(wia + i), __ldg(wib + i))));
        }
    }
    FFT::run(v, s, t, a.btw + fft_twiddle_offset(LZ));
    __syncthreads();
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int q = (t + T * i) << u.logR;
        zs[pidx(q + ra)] = lane_a(v[i]);
        zs[pidx(q + rb)] = lane_b(v[i]);
    }
    __syncthreads();
    if (!live) return;
    float2* Xr = a.X + it.out_off;
    const float2* wp = tab + R * T + R * E;
    const float2 w0 = __ldg(wp + lt);
    int kj = 0;
#pragma unroll 4
    for (int k = lt; k <= H / 2; k += PT, kj += PT)
        unpack_pair(Xr, k, H, zs[pidx(k)], zs[pidx((H - k) & (H - 1))], cmul(w0, __ldg(wp + kj)));
}

// mode 1: G residue pairs g0 .. g0 + G - 1 of one trace
template <int LZ>
__device__ __forceinline__ void fft_queue_pairs(const FftQueueArgs& a, const FftUnit& u, float4* smem4) {
    using FFT = BlockFFT<LZ, false, C2>;
    constexpr int E = FFT::E, T = FFT::T;
    const int R = 1 << u.logR;
    const int H = R * LZ;
    const int tid = threadIdx.x;
    const int gl = tid / T;
    const int t = tid - gl * T;
    const int g = u.g0 + gl;
    const bool live = gl < u.count;                            // pairs in this unit
    const RaggedItem it = a.items[u.item];
    const int n = it.n;
    float4* s = smem4 + gl * padded_len(LZ);
    const float2* tab = u.tab;
    const int ra = live ? g : 0;

    C2 v[E];
    {
        // w_H^{r m} = w_H^{r t} w_H^{r T i} for r = g (both lanes; pair 0:
        // lane a residue 0, lane b residue R/2)
        const int rw = g == 0 ? R / 2 : ra;
        const float2 wt = __ldg(tab + rw * T + t);
        const float2* wi = tab + R * T + rw * E;
        const float* xr = a.x + it.x_off;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int m = t + T * i;
            float2 z = make_float2(0.f, 0.f);
            if (live && 2 * m < n) z.x = __ldg(xr + 2 * m);
            if (live && 2 * m + 1 < n) z.y = __ldg(xr + 2 * m + 1);
            const float2 w = cmul(wt, __ldg(wi + i));
            if (g != 0) {
                const float P = z.x * w.x, Q = z.y * w.y, S = z.x * w.y, U = z.y * w.x;
                v[i] = C2{make_float2(P - Q, P + Q), make_float2(S + U, S - U)};
            } else {
                v[i] = C2{make_float2(z.x, fmaf(z.x, w.x, -z.y * w.y)), make_float2(z.y, fmaf(z.x, w.y, z.y * w.x))};
            }
        }
    }
    FFT::run(v, s, t, a.btw + fft_twiddle_offset(LZ));
    __syncthreads();
    float2* z0 = reinterpret_cast<float2*>(s);
    float2* z4 = z0 + padded_len(LZ);
    if (g == 0) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            z0[pidx(t + T * i)] = lane_a(v[i]);
            z4[pidx(t + T * i)] = lane_b(v[i]);
        }
    }
    __syncthreads();
    if (!live) return;
    float2* Xr = a.X + it.out_off;
    const float2* wp = tab + R * T + R * E;                    // w_{2H}^k, k <= H/2
    const float2 wb0 = cscale(__ldg(wp + R * t + g), 0.5f);
    const float2 wb4 = cscale(__ldg(wp + R * t + R / 2), 0.5f);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        // w_{2H}^{R (t + T i) + g} = w_{2H}^{R t + g} e^{-j pi i/16} (R T = H/16)
        const float ci = i <= 8 ? cos_pi16(i) : -cos_pi16(16 - i);
        const float si = i <= 8 ? cos_pi16(8 - i) : cos_pi16(i - 8);
        const float2 ei = make_float2(ci, -si);
        const int q = t + T * i;
        if (g != 0) {
            const float2 wh = cmul(wb0, ei);
            Xr[R * q + g] = unpack_fwd(lane_a(v[i]), lane_b(v[i]), wh);
            Xr[H - (R * q + g)] = unpack_mirror(lane_a(v[i]), lane_b(v[i]), wh);
        } else {
            const float2 B0 = z0[pidx((LZ - q) & (LZ - 1))], B4 = z4[pidx(LZ - 1 - q)];
            Xr[R * q] = unpack_fwd(lane_a(v[i]), make_float2(B0.x, -B0.y), cmul(wb0, ei));
            Xr[R * q + R / 2] = unpack_fwd(lane_b(v[i]), make_float2(B4.x, -B4.y), cmul(wb4, ei));
        }
    }
    if (g == 0 && t == 0) {
        const float2 Z0 = lane_a(v[0]);
        Xr[H] = make_float2(Z0.x - Z0.y, 0.f);
    }
}

// mode 2: one whole trace too long for the CTA's shared memory.  The residue
// pairs (g, g + R/2) run in rounds of G = 512/(LZ/16); each round writes its
// Z values to this CTA's workspace (H complex values, residue-major, so the
// stores are coalesced; it stays in L2), and after the last round the CTA
// unpacks every pair (k, H - k) from the workspace with coalesced stores of X.
template <int LZ>
__device__ __forceinline__ void fft_queue_ws(const FftQueueArgs& a, const FftUnit& u, float4* smem4) {
    using FFT = BlockFFT<LZ, false, C2>;
    constexpr int E = FFT::E, T = FFT::T;
    constexpr int G = kFftQueueThreads / T;
    const int logR = u.logR;
    const int R = 1 << logR;
    const int H = R * LZ;
    const int tid = threadIdx.x;
    const int gl = tid / T;
    const int t = tid - gl * T;
    const RaggedItem it = a.items[u.item];
    const int n = it.n;
    float4* s = smem4 + gl * padded_len(LZ);
    const float2* tab = u.tab;
    float2* ws = a.ws + (size_t)blockIdx.x * a.ws_per_cta;
    const float* xr = a.x + it.x_off;
    for (int g0 = 0; g0 < R / 2; g0 += G) {
        const int ra = g0 + gl, rb = ra + R / 2;
        const bool on = ra < R / 2;
        const int rra = on ? ra : 0, rrb = on ? rb : R / 2;
        C2 v[E];
        const C2 wt = c2(__ldg(tab + rra * T + t), __ldg(tab + rrb * T + t));
        const float2* wia = tab + R * T + rra * E;
        const float2* wib = tab + R * T + rrb * E;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int m = t + T * i;
            float re = 0.f, im = 0.f;
            if (2 * m < n) re = __ldg(xr + 2 * m);
            if (2 * m + 1 < n) im = __ldg(xr + 2 * m + 1);
            v[i] = cmul(make_float2(re, im), cmul(wt, c2(__ldg(wia + i), __ldg(wib + i))));
        }
        FFT::run(v, s, t, a.btw + fft_twiddle_offset(LZ));
        if (on) {
            float2* za = ws + (size_t)ra * LZ + t;
            float2* zb = ws + (size_t)rb * LZ + t;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                za[T * i] = lane_a(v[i]);
                zb[T * i] = lane_b(v[i]);
            }
        }
        __syncthreads();                                         // s is reused by the next round
    }
    // (the barrier above also makes every thread's workspace stores visible)
    float2* Xr = a.X + it.out_off;
    const float2* wp = tab + R * T + R * E;                      // w_{2H}^k, k <= H/2
    const int mask = R - 1;
#pragma unroll 4
    for (int k = tid; k <= H / 2; k += kFftQueueThreads) {
        const int km = (H - k) & (H - 1);
        const float2 A = ws[(size_t)(k & mask) * LZ + (k >> logR)];
        const float2 B = ws[(size_t)(km & mask) * LZ + (km >> logR)];
        unpack_pair(Xr, k, H, A, B, __ldg(wp + k));
    }
}

__global__ void __launch_bounds__(kFftQueueThreads, 2) k_fft_queue(FftQueueArgs a) {
    extern __shared__ float4 smem4[];
    __shared__ int s_unit;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_unit = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int ui = s_unit;
        if (ui >= a.nunits) return;
        const FftUnit u = a.units[ui];
#define SPEC_QUEUE_CASE(lz)                                                    \
    case lz:                                                                   \
        if (u.mode == 0) fft_queue_full<lz>(a, u, smem4);                      \
        else if (u.mode == 1) fft_queue_pairs<lz>(a, u, smem4);                \
        else fft_queue_ws<lz>(a, u, smem4);                                    \
        break;
        switch (u.LZ) {
            SPEC_QUEUE_CASE(16) SPEC_QUEUE_CASE(32) SPEC_QUEUE_CASE(64) SPEC_QUEUE_CASE(128)
            SPEC_QUEUE_CASE(256) SPEC_QUEUE_CASE(512) SPEC_QUEUE_CASE(1024) SPEC_QUEUE_CASE(2048)
            SPEC_QUEUE_CASE(4096)
            default: break;
        }
#undef SPEC_QUEUE_CASE
    }
}

// 4096 packed pairs of C2 values in padded layout, plus slack for the
// whole-trace staging (F (padded_len(H) + 2) float2 per unit)
size_t fft_queue_smem() { return (size_t)kFftQueueThreads * 17 * sizeof(float4) + 1024; }

cudaError_t fft_queue_launch(const RaggedItem* items, const FftUnit* units, int nunits, unsigned* counter,
                             const float* x_pool, const float2* btw, float2* X_pool, float2* ws, int64_t ws_per_cta,
                             int ctas, cudaStream_t st) {
    if (nunits == 0) return cudaSuccess;
    const size_t smem = fft_queue_smem();
    cudaError_t e = cudaFuncSetAttribute(k_fft_queue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    FftQueueArgs a = {};
    a.items = items; a.units = units; a.nunits = nunits; a.counter = counter;
    a.x = x_pool; a.X = X_pool; a.btw = btw; a.ws = ws; a.ws_per_cta = ws_per_cta;
    k_fft_queue<<<(unsigned)std::max(1, std::min(ctas, nunits)), kFftQueueThreads, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pruned complex FFT with a rotated store: Y[(j + shift) mod K] = U[j],
// U = FFT_K of u[0 .. nin-1] zero-padded to K.  The same residue
// decomposition as above (R = K/LZ pre-twiddled LZ-point FFTs, a cluster of
// C CTAs when K > 8192), but the input is complex and each CTA stores its
// own contiguous chunk of U, so distributed shared memory is only written.
// Used by the Zoom FFT when its K-point FFT does not fit one CTA (the
// ascending-frequency order of Section 2.2 is the rotation by K/2).
struct C2cArgs {
    const float2* u;
    int64_t ld_u;
    int nin;
    int64_t batch;
    int K, logR, Rc, C, F, logChunk, trace_smem, shift;
    const float2* tw;
    const float2* tab;    // [w_K^{r t}: R x T][w_K^{r T i}: R x E]
    float2* X;
    int64_t ld_X;
    const RaggedItem* items;   // ragged batch: nin = lout, u / X offsets (else null)
};

template <int E, int T>
__device__ __forceinline__ void c2c_epilogue(const C2cArgs& a, float2 (&v)[E]);

template <int LZ>
__global__ void __launch_bounds__(1024, 1) k_fft_c2c_pruned(C2cArgs a) {
    using FFT = BlockFFT<LZ, false>;
    constexpr int E = FFT::E;
    constexpr int T = FFT::T;
    extern __shared__ float2 smem[];

    const int per_trace = a.Rc * T;
    const int tid = threadIdx.x;
    const int f = tid / per_trace;
    const int lt = tid - f * per_trace;
    const int rl = lt / T;
    const int t = lt - rl * T;
    const int rank = a.C > 1 ? (int)(blockIdx.x % a.C) : 0;
    const int64_t b = (int64_t)(blockIdx.x / a.C) * a.F + f;
    const bool live = b < a.batch;
    int nin = a.nin;
    int64_t uo = (live ? b : 0) * a.ld_u;
    if (a.items && live) {
        const RaggedItem& it = a.items[b];
        uo = it.u_off;
        nin = it.lout;
    }
    const int R = 1 << a.logR;
    const int r = rank * a.Rc + rl;
    float2* zs = smem + f * a.trace_smem;
    float2* s = zs + rl * padded_len(LZ);

    float2 v[E];
    {
        const float2 wt = __ldg(a.tab + r * T + t);
        const float2* wi = a.tab + R * T + r * E;
        const float2* ur = a.u + uo;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int m = t + T * i;
            const float2 z = (live && m < nin) ? __ldg(ur + m) : make_float2(0.f, 0.f);
            v[i] = cmul(z, cmul(wt, __ldg(wi + i)));
        }
    }
    FFT::run(v, s, t, a.tw);
    c2c_epilogue<E, T>(a, v);     // placement re-derived: only v[] is live across the FFT
}

template <int E, int T>
__device__ __forceinline__ void c2c_epilogue(const C2cArgs& a, float2 (&v)[E]) {
    extern __shared__ float2 smem[];
    const int per_trace = a.Rc * T;
    const int tid = (int)opaque_tid();
    const int f = tid / per_trace;
    const int lt = tid - f * per_trace;
    const int rl = lt / T;
    const int t = lt - rl * T;
    const unsigned cta = opaque_ctaid();
    const int rank = a.C > 1 ? (int)(cta % a.C) : 0;
    const int64_t b = (int64_t)(cta / a.C) * a.F + f;
    const bool live = b < a.batch;
    const int64_t Xo = !live ? 0 : a.items ? a.items[b].out_off : b * a.ld_X;
    const int r = rank * a.Rc + rl;
    float2* zs = smem + f * a.trace_smem;
    const int chunk = 1 << a.logChunk;
    if (a.C > 1) {
        // several CTAs per transform: each writes its own residues' outputs
        // Y[(R q + r + shift) mod K] directly -- runs of Rc consecutive
        // outputs at stride R, no exchange between the CTAs
        if (live) {
            float2* Xr = a.X + Xo;
#pragma unroll
            for (int i = 0; i < E; ++i) Xr[((((t + T * i) << a.logR) + r) + a.shift) & (a.K - 1)] = v[i];
        }
        return;
    }
    // one CTA: stage U in natural order, then contiguous rotated stores
    __syncthreads();
#pragma unroll
    for (int i = 0; i < E; ++i) zs[pidx(((t + T * i) << a.logR) + r)] = v[i];
    __syncthreads();
    if (live) {
        float2* Xr = a.X + Xo;
        for (int j = lt; j < chunk; j += per_trace) Xr[(j + a.shift) & (a.K - 1)] = zs[pidx(j)];
    }
}

using C2cKernel = void (*)(C2cArgs);

static C2cKernel c2c_kernel_for(int LZ) {
    switch (LZ) {
        case 16: return k_fft_c2c_pruned<16>;
        case 32: return k_fft_c2c_pruned<32>;
        case 64: return k_fft_c2c_pruned<64>;
        case 128: return k_fft_c2c_pruned<128>;
        case 256: return k_fft_c2c_pruned<256>;
        case 512: return k_fft_c2c_pruned<512>;
        case 1024: return k_fft_c2c_pruned<1024>;
        case 2048: return k_fft_c2c_pruned<2048>;
        case 4096: return k_fft_c2c_pruned<4096>;
        case 8192: return k_fft_c2c_pruned<8192>;
        default: return nullptr;
    }
}

bool c2c_plan(int64_t batch, int64_t nin, int64_t K, FftPlan* p, std::string* why) {
    *p = FftPlan();
    int64_t LZ = std::max<int64_t>(16, next_pow2(nin));
    LZ = std::min<int64_t>(LZ, K);
    if (K < 16 || LZ > kTile) {
        *why = "pruned FFT: needs 16 <= K and at most 8192 nonzero inputs";
        return false;
    }
    const int64_t R = K / LZ;
    // up to 16384 points per CTA (1024 threads) for long residue FFTs; a
    // larger K spreads the residues over C CTAs that store independently
    const int64_t tile = LZ >= 2048 ? 2 * kTile : kTile;
    const int64_t C = std::max<int64_t>(1, K / tile);
    if (C > 8) {
        *why = "pruned FFT: K above 65536 needs the multi-pass path";
        return false;
    }
    p->H = (int)K;
    p->LZ = (int)LZ;
    p->R = (int)R;
    p->C = (int)C;
    p->Rc = (int)(R / C);
    p->E = 16;
    p->T = (int)LZ / 16;
    const int per_trace = p->Rc * p->T;
    p->F = 1;
    if (C == 1) p->F = (int)std::min<int64_t>(std::max(1, 256 / per_trace), std::max<int64_t>(1, batch));
    p->trace_smem = C > 1 ? p->Rc * padded_len((int)LZ) : std::max(p->Rc * padded_len((int)LZ), padded_len((int)K));
    p->threads = p->F * per_trace;
    p->smem = (size_t)p->F * p->trace_smem * sizeof(float2);
    return true;
}

int c2c_table_entries(const FftPlan& p) { return p.R * p.T + p.R * p.E; }

void c2c_fill_table(const FftPlan& p, float2* host) {
    const double two_pi = 6.283185307179586476925286766559;
    const int64_t K = p.H;
    auto w = [&](int64_t num) {
        const double ang = two_pi * (double)(num % K) / (double)K;
        return make_float2((float)std::cos(ang), (float)-std::sin(ang));
    };
    float2* o = host;
    for (int r = 0; r < p.R; ++r)
        for (int t = 0; t < p.T; ++t) *o++ = w((int64_t)r * t);
    for (int r = 0; r < p.R; ++r)
        for (int i = 0; i < p.E; ++i) *o++ = w((int64_t)r * p.T * i);
}

cudaError_t c2c_launch(const FftPlan& p, const float2* u, int64_t ld_u, int nin, int64_t batch, int shift,
                       const float2* tw, const float2* tab, float2* X, int64_t ld_X, cudaStream_t st,
                       const RaggedItem* items) {
    if (batch == 0) return cudaSuccess;
    C2cKernel k = c2c_kernel_for(p.LZ);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    C2cArgs a = {};
    a.u = u; a.ld_u = ld_u; a.nin = nin; a.batch = batch;
    a.K = p.H; a.logR = ilog2(p.R); a.Rc = p.Rc; a.C = p.C; a.F = p.F;
    a.logChunk = ilog2(p.H / p.C); a.trace_smem = p.trace_smem; a.shift = shift;
    a.tw = tw; a.tab = tab; a.X = X; a.ld_X = ld_X; a.items = items;
    const int64_t groups = (batch + p.F - 1) / p.F;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(groups * p.C));
    cfg.blockDim = dim3(p.threads);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = st;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;            // the CTAs of one transform never communicate
    return cudaLaunchKernelEx(&cfg, k, a);
}

// n_fft == 1: the single bin is x[0].
__global__ void k_fft_len1(const float* x, int64_t batch, int64_t ld_x, float2* X, int64_t ld_X) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < batch) X[b * ld_X] = make_float2(x[b * ld_x], 0.f);
}

using FftKernel = void (*)(FftArgs);

static FftKernel fft_kernel2_for(int LZ) {
    switch (LZ) {
        case 16: return k_fft_real_padded2<16>;
        case 32: return k_fft_real_padded2<32>;
        case 64: return k_fft_real_padded2<64>;
        case 128: return k_fft_real_padded2<128>;
        case 256: return k_fft_real_padded2<256>;
        case 512: return k_fft_real_padded2<512>;
        case 1024: return k_fft_real_padded2<1024>;
        case 2048: return k_fft_real_padded2<2048>;
        case 4096: return k_fft_real_padded2<4096>;
        default: return nullptr;
    }
}

// (LZ, R) pairs with a compiled fixed two-lane kernel.  Measured on GB300:
// 65536 traces of 1024 samples to 8192 points (LZ 512, R 8) 801 -> 775 us;
// 4096 traces of 2048 samples to 16384 points (LZ 1024, R 8) 109 -> 113 us
// (spec_fft times the variants of a shape and keeps the faster).
static FftKernel fft_kernel_fixed_for(int LZ, int R) {
#define SPEC_FIXED(lz, r) if (LZ == lz && R == r) return k_fft_real_padded2r<lz, r>;
    SPEC_FIXED(256, 8) SPEC_FIXED(512, 8) SPEC_FIXED(1024, 8)
    SPEC_FIXED(512, 4) SPEC_FIXED(1024, 4) SPEC_FIXED(2048, 4)
    SPEC_FIXED(256, 16) SPEC_FIXED(512, 16)
    SPEC_FIXED(1024, 2) SPEC_FIXED(2048, 2) SPEC_FIXED(4096, 2)
#undef SPEC_FIXED
    return nullptr;
}

// (LZ, R) pairs with a compiled fused-unpack kernel (three-pass BlockFFT,
// R/2 LZ/16 threads per trace a multiple of 128)
static FftKernel fft_kernel_fused_for(int LZ, int R, bool tma = false, int fold = 1) {
    if (fold == 2) {
        // folded input (traces of up to 2 LZ sample pairs), plain grid only
        if (tma) return nullptr;
        if (LZ == 512 && R == 8) return k_fft_real_fused<512, 8, 2>;
        if (LZ == 512 && R == 16) return k_fft_real_fused<512, 16, 2>;
        return nullptr;
    }
    if (fold != 1) return nullptr;
#define SPEC_FUSED(lz, r) if (LZ == lz && R == r) return tma ? k_fft_real_fused_tma<lz, r> : k_fft_real_fused<lz, r>;
    SPEC_FUSED(512, 8) SPEC_FUSED(512, 16) SPEC_FUSED(1024, 4) SPEC_FUSED(1024, 8)
#undef SPEC_FUSED
    return nullptr;
}
bool fft_fused_available(int LZ, int R, int fold) { return fft_kernel_fused_for(LZ, R, false, fold) != nullptr; }

// (LZ, R) pairs with a compiled cluster kernel (one trace per cluster of
// R LZ/8192 CTAs)
static FftKernel fft_kernel_cluster_for(int LZ, int R) {
#define SPEC_CLUSTER(lz, r) if (LZ == lz && R == r) return k_fft_real_cluster<lz, r>;
    SPEC_CLUSTER(4096, 4) SPEC_CLUSTER(4096, 8) SPEC_CLUSTER(4096, 16)
    SPEC_CLUSTER(2048, 8) SPEC_CLUSTER(2048, 16) SPEC_CLUSTER(2048, 32)
    SPEC_CLUSTER(1024, 16) SPEC_CLUSTER(1024, 32) SPEC_CLUSTER(1024, 64)
#undef SPEC_CLUSTER
    return nullptr;
}
constexpr size_t kClusterSmem = (size_t)(pidx8(kClusterRun) + 2) * sizeof(float2);

static FftKernel fft_kernel_for(int LZ, int emax) {
    if (emax == 32) {
        switch (LZ) {
            case 512: return k_fft_real_padded<512, 32>;
            case 1024: return k_fft_real_padded<1024, 32>;
            case 8192: return k_fft_real_padded<8192, 32>;
            default: return nullptr;
        }
    }
    switch (LZ) {
        case 1: return k_fft_real_padded<1, 16>;
        case 2: return k_fft_real_padded<2, 16>;
        case 4: return k_fft_real_padded<4, 16>;
        case 8: return k_fft_real_padded<8, 16>;
        case 16: return k_fft_real_padded<16, 16>;
        case 32: return k_fft_real_padded<32, 16>;
        case 64: return k_fft_real_padded<64, 16>;
        case 128: return k_fft_real_padded<128, 16>;
        case 256: return k_fft_real_padded<256, 16>;
        case 512: return k_fft_real_padded<512, 16>;
        case 1024: return k_fft_real_padded<1024, 16>;
        case 2048: return k_fft_real_padded<2048, 16>;
        case 4096: return k_fft_real_padded<4096, 16>;
        case 8192: return k_fft_real_padded<8192, 16>;
        default: return nullptr;
    }
}

// Elements per thread of the residue FFTs.  Radix-32 passes save one
// shared-memory exchange at 512, 1024 and 8192 points, but at 1024 points
// (4096 traces x 2048 samples to 16384) they measured slower than radix 16
// (150 vs 144 us: half the occupancy at 128 registers), so radix 16 is used;
// the radix-32 kernels stay available through SPEC_FFT_EMAX=32.
int fft_emax_for(int LF) {
    static const int forced = [] {
        const char* e = std::getenv("SPEC_FFT_EMAX");
        return e ? std::atoi(e) : 16;
    }();
    return (forced == 32 && (LF == 512 || LF == 1024 || LF == 8192)) ? 32 : 16;
}

bool fft_plan(int64_t batch, int64_t n, int64_t n_fft, FftPlan* p, std::string* why, bool allow_cluster) {
    *p = FftPlan();
    if (n_fft == 1) return true;
    const int64_t H = n_fft / 2;
    int64_t LZ = next_pow2((n + 1) / 2);
    LZ = std::max<int64_t>(LZ, std::min<int64_t>(16, H));
    LZ = std::min<int64_t>(LZ, H);
    if (LZ > kTile) {
        *why = "padded FFT: more than 16384 samples per trace needs the multi-pass path";
        return false;
    }
    const int64_t R = H / LZ;
    // Points per CTA: 16384 (1024 threads, one CTA per SM) when the residue
    // FFTs are long, which keeps 32768-point transforms in one CTA and halves
    // the CTAs of 65536-point ones; 8192 otherwise (measured on GB300: 79 vs
    // 101 ns per 4096-sample trace to 32768 points, 213 vs 191 ns per
    // 2048-sample trace to 65536 points).
    const int64_t tile = LZ >= 2048 ? 2 * kTile : kTile;
    const int64_t C = std::max<int64_t>(1, H / tile);
    if (C > 8) {
        *why = "padded FFT: n_fft above 131072 needs the multi-pass path";
        return false;
    }
    p->emax = fft_emax_for((int)LZ);
    const int E = LZ < p->emax ? (int)LZ : p->emax;
    const int T = (int)LZ / E;
    p->H = (int)H;
    p->LZ = (int)LZ;
    p->R = (int)R;
    p->C = (int)C;
    p->Rc = (int)(R / C);
    p->E = E;
    p->T = T;
    // C > 1: CTAs own residue pairs and unpack alone (no cluster) when every
    // CTA can hold whole pairs; otherwise a cluster exchanges Z through
    // distributed shared memory
    p->paired = C > 1 && (p->Rc % 2 == 0 || (p->Rc == 1 && R == 2));
    p->dual = p->Rc >= 2 && LZ >= 16 && LZ <= 4096 && p->emax == 16 && !p->paired && (p->Rc / 2) * T <= 256;
    p->fixed = p->dual && C == 1 && fft_kernel_fixed_for((int)LZ, (int)R) != nullptr;
    p->clustered = allow_cluster && fft_kernel_cluster_for((int)LZ, (int)R) != nullptr && fft_emax_for((int)LZ) == 16;
    if (p->clustered) {
        // one cluster of R LZ/8192 CTAs per trace, 256 threads each
        p->C = (int)(R * LZ / kClusterRun);
        p->Rc = (int)(R / p->C);
        p->paired = p->dual = p->fixed = false;
        p->E = 16;
        p->T = (int)LZ / 16;
        p->F = 1;
        p->trace_smem = (int)(kClusterSmem / sizeof(float2));
        p->threads = 256;
        p->smem = kClusterSmem;
        return true;
    }
    const int per_trace = p->dual ? (p->Rc / 2) * T : p->Rc * T;
    p->F = 1;
    if (C == 1) {
        int64_t F = std::max<int64_t>(1, 256 / per_trace);
        F = std::min<int64_t>(F, std::max<int64_t>(1, batch));
        p->F = (int)F;
    }
    const int chunk = (int)(H / C);
    // the cluster staging uses padded slots 0 .. chunk (pidx(chunk) = padded_len(chunk))
    p->trace_smem = std::max(p->Rc * padded_len((int)LZ), padded_len(chunk) + 1);
    p->trace_smem += p->trace_smem & 1;       // keep float4 views 16-byte aligned
    p->threads = p->F * per_trace;
    p->smem = (size_t)p->F * p->trace_smem * sizeof(float2);
    return true;
}

int fft_table_entries(const FftPlan& p) {
    if (p.clustered) return 2 * (cluster_tw4_index(p.H) + fft_twiddle_entries(p.LZ));
    if (p.fused) return fused_entries(p.LZ, p.R, p.fold);
    const int generic = p.R * p.T + p.R * p.E + p.H / 2 + 1;
    if (!p.fixed) return generic;
    // + packed pre-twiddles [R/2][LZ] and BlockFFT<LZ> twiddles, float4 each
    return 2 * (fixed_tw4_index(p.LZ, p.R) + fft_twiddle_entries(p.LZ));
}

void fft_fill_table(const FftPlan& p, float2* host) {
    const double two_pi = 6.283185307179586476925286766559;
    const int64_t H = p.H;
    auto w = [&](int64_t num, int64_t den) {     // e^{-j 2 pi num/den}, exact reduction
        const double ang = two_pi * (double)(num % den) / (double)den;
        return make_float2((float)std::cos(ang), (float)-std::sin(ang));
    };
    auto tw4_fill = [&](float4* t4) {
        // BlockFFT<LZ> twiddles of the radix-16 layout as packed pairs (c, c, s, s)
        const int lg = ilog2(p.LZ), npb = lg / 4, rem = 1 << (lg % 4);
        const int npass = npb + (rem > 1 ? 1 : 0);
        int ns = 1;
        for (int q = 0; q < npass; ++q) {
            const int Rq = q < npb ? 16 : rem;
            if (q >= 1)
                for (int r = 1; r < Rq; ++r)
                    for (int k = 0; k < ns; ++k) {
                        const float2 e = w((int64_t)r * k, (int64_t)ns * Rq);
                        t4[ns - 16 + (r - 1) * ns + k] = make_float4(e.x, e.x, e.y, e.y);
                    }
            ns *= Rq;
        }
    };
    if (p.clustered) {
        for (int64_t k = 0; k <= H / 2; ++k) host[k] = w(k, 2 * H);
        float2* pre = host + cluster_pre_offset(p.H);
        for (int g = 0; g < p.R / 2; ++g)
            for (int m = 0; m < p.LZ; ++m)
                pre[(int64_t)g * p.LZ + m] = w((int64_t)(g == 0 ? p.R / 2 : g) * m, H);
        tw4_fill(reinterpret_cast<float4*>(host) + cluster_tw4_index(p.H));
        return;
    }
    if (p.fused) {
        // pre4: lanes 2g and 2g + 1 at m; BlockFFT twiddles; the unpack bases
        float4* t4 = reinterpret_cast<float4*>(host);
        for (int g = 0; g < p.R / 2; ++g)
            for (int m = 0; m < p.LZ; ++m) {
                const float2 wa = w((int64_t)(2 * g) * m, H), wb = w((int64_t)(2 * g + 1) * m, H);
                t4[(int64_t)g * p.LZ + m] = make_float4(wa.x, wb.x, wa.y, wb.y);
            }
        {
            // BlockFFT<LZ> twiddles as (c, s): the packed form, then repacked
            std::vector<float4> t4tw((size_t)fft_twiddle_entries(p.LZ));
            tw4_fill(t4tw.data());
            float2* d2 = host + fused_tw2_index(p.LZ, p.R, p.fold);
            for (size_t e = 0; e < t4tw.size(); ++e) d2[e] = make_float2(t4tw[e].x, t4tw[e].z);
        }
        const int PT = (p.R / 2) * (p.LZ / 16);
        const int NS = p.LZ / (1 << (ilog2(p.LZ) % 4));  // span of the fused last pass
        if (p.fold == 2) {
            // fold4: w_R^{2g}, w_R^{2g+1} (= w_H^{LZ r}), packed like pre4
            float4* f4 = t4 + fused_fold4_index(p.LZ, p.R);
            for (int g = 0; g < p.R / 2; ++g) {
                const float2 ca = w(2 * g, p.R), cb = w(2 * g + 1, p.R);
                f4[g] = make_float4(ca.x, cb.x, ca.y, cb.y);
            }
        }
        float4* ub = t4 + fused_ub4_index(p.LZ, p.R, p.fold);
        float2* um = host + fused_um_index(p.LZ, p.R, p.fold);
        for (int lt = 0; lt < PT; ++lt) {
            const int r = lt % p.R, q0 = lt / p.R;
            const float2 wk = w(lt, 2 * H), wq = w(q0, p.LZ);
            ub[lt] = make_float4(0.5f * wk.x, 0.5f * wk.y, wq.x, wq.y);
            um[lt] = w(r > 0 ? NS - 1 - q0 : NS - q0, p.LZ);
        }
        return;
    }
    float2* o = host;
    for (int r = 0; r < p.R; ++r)
        for (int t = 0; t < p.T; ++t) *o++ = w((int64_t)r * t, H);
    for (int r = 0; r < p.R; ++r)
        for (int i = 0; i < p.E; ++i) *o++ = w((int64_t)r * p.T * i, H);
    for (int64_t k = 0; k <= H / 2; ++k) *o++ = w(k, 2 * H);
    if (!p.fixed) return;
    // packed two-lane pre-twiddles: lanes g and g + R/2 at m
    float4* o4 = reinterpret_cast<float4*>(host) + fixed_pre4_index(p.LZ, p.R);
    for (int g = 0; g < p.R / 2; ++g)
        for (int m = 0; m < p.LZ; ++m) {
            const float2 wa = w((int64_t)g * m, H), wb = w((int64_t)(g + p.R / 2) * m, H);
            *o4++ = make_float4(wa.x, wb.x, wa.y, wb.y);
        }
    tw4_fill(reinterpret_cast<float4*>(host) + fixed_tw4_index(p.LZ, p.R));
}

bool fft_fused_tma_ok(const FftPlan& p, const float* x, int n, int64_t ld_x) {
    return p.fused && p.fold == 1 && fft_kernel_fused_for(p.LZ, p.R, true) != nullptr && n == 2 * p.LZ &&
           (reinterpret_cast<uintptr_t>(x) & 15) == 0 && (ld_x & 3) == 0;
}

cudaError_t fft_fused_tma_launch(const FftPlan& p, const float* x, int64_t batch, int64_t ld_x, const float2* tab,
                                 float2* X, int64_t ld_X, unsigned* status, uint64_t timeout_ns, int sms,
                                 cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    FftKernel kf = fft_kernel_fused_for(p.LZ, p.R, true);
    if (!kf) return cudaErrorInvalidValue;
    const int PT = (p.R / 2) * (p.LZ / 16);
    const int F = std::max(1, 256 / PT);
    const size_t smem = fused_tma_smem(p.LZ, p.R);
    cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    FftArgs a = {};
    a.x = x; a.batch = batch; a.n = 2 * p.LZ; a.ld_x = ld_x;
    a.H = p.H; a.logR = ilog2(p.R); a.Rc = p.Rc; a.C = 1; a.F = F;
    a.tab = tab; a.X = X; a.ld_X = ld_X;
    a.status = status;
    a.timeout_ns = timeout_ns;
    const int64_t groups = (batch + F - 1) / F;
    const int64_t grid = std::min<int64_t>(groups, 2 * (int64_t)std::max(1, sms));
    kf<<<(unsigned)grid, F * PT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t fft_launch(const FftPlan& p, const float* x, int64_t batch, int n, int64_t ld_x,
                       const float2* tw, const float2* tab, float2* X, int64_t ld_X, cudaStream_t st,
                       int lanes, const RaggedItem* items) {
    if (batch == 0) return cudaSuccess;
    if (p.H == 0) {   // n_fft == 1
        k_fft_len1<<<(unsigned)((batch + 255) / 256), 256, 0, st>>>(x, batch, ld_x, X, ld_X);
        return cudaGetLastError();
    }
    if (p.clustered) {
        FftKernel kc = fft_kernel_cluster_for(p.LZ, p.R);
        cudaError_t e = cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusterSmem);
        if (e != cudaSuccess) return e;
        FftArgs a = {};
        a.x = x; a.batch = batch; a.n = n; a.ld_x = ld_x;
        a.H = p.H; a.logR = ilog2(p.R); a.Rc = p.Rc; a.C = p.C; a.F = 1;
        a.tab = tab; a.X = X; a.ld_X = ld_X; a.items = items;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(batch * p.C));
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = kClusterSmem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = p.C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kc, a);
    }
    const bool dual = p.dual && lanes != 1;
    if (dual && p.fused) {
        FftKernel kf = fft_kernel_fused_for(p.LZ, p.R, false, p.fold);
        if (!kf) return cudaErrorInvalidValue;
        const int PT = (p.R / 2) * (p.LZ / 16);
        const int F = std::max(1, 256 / PT);
        const size_t smem = (size_t)F * fused_trace_smem(p.LZ, p.R) * sizeof(float2);
        cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        FftArgs a = {};
        a.x = x; a.batch = batch; a.n = n; a.ld_x = ld_x;
        a.H = p.H; a.logR = ilog2(p.R); a.Rc = p.Rc; a.C = 1; a.F = F;
        a.tab = tab; a.X = X; a.ld_X = ld_X; a.items = items;
        kf<<<(unsigned)((batch + F - 1) / F), F * PT, smem, st>>>(a);
        return cudaGetLastError();
    }
    if (dual && p.fixed) {
        // compile-time (LZ, R): 256 threads, 256 / (R/2 LZ/16) traces per CTA
        FftKernel kf = fft_kernel_fixed_for(p.LZ, p.R);
        const int PT = (p.R / 2) * (p.LZ / 16);
        const int F = std::max(1, 256 / PT);
        const size_t smem = (size_t)F * (padded_len(p.H) + 2) * sizeof(float2);
        cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        FftArgs a = {};
        a.x = x; a.batch = batch; a.n = n; a.ld_x = ld_x;
        a.H = p.H; a.logR = ilog2(p.R); a.Rc = p.Rc; a.C = 1; a.F = F;
        a.tab = tab; a.X = X; a.ld_X = ld_X; a.items = items;
        kf<<<(unsigned)((batch + F - 1) / F), F * PT, smem, st>>>(a);
        return cudaGetLastError();
    }
    FftKernel k = dual ? fft_kernel2_for(p.LZ) : fft_kernel_for(p.LZ, p.emax);
    if (!k) return cudaErrorInvalidValue;
    FftArgs a = {};
    a.x = x; a.batch = batch; a.n = n; a.ld_x = ld_x;
    a.H = p.H; a.logR = ilog2(p.R); a.Rc = p.Rc; a.C = p.C;
    a.logChunk = ilog2(p.H / p.C); a.trace_smem = p.trace_smem;
    a.tw = tw; a.tab = tab;
    a.X = X; a.ld_X = ld_X; a.items = items;
    a.paired = p.paired ? 1 : 0;
    const int per_trace = dual ? (p.Rc / 2) * p.T : p.Rc * p.T;
    int F = 1;
    if (p.C == 1) F = (int)std::min<int64_t>(std::max(1, 256 / per_trace), std::max<int64_t>(1, batch));
    a.F = F;
    const size_t smem = (size_t)F * p.trace_smem * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t groups = (batch + F - 1) / F;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(groups * p.C));
    cfg.blockDim = dim3(F * per_trace);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    cfg.attrs = attr;
    cfg.numAttrs = 0;
    if (p.C > 1 && !p.paired) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = p.C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace spec
