// k_long.cu -- multi-pass transforms for traces too long for one CTA or one
// cluster: the zero-padded FFT of Section 2.1 (Eq. 2) beyond N_FFT = 131072
// or 16384 samples, and Bluestein's chirp-z transform of Section 2.3
// (Eq. 13-15) beyond L = 16384.
//
// A P-point FFT is split as P = P1 x P2 with rows of P2 = 512 points (the
// "four-step" factorisation):
//
//   m = P2 m1 + m2,  k = k1 + P1 k2,
//   Y[k1 + P1 k2] = sum_m2 w_P2^{m2 k2} [ w_P^{m2 k1} sum_m1 y[P2 m1 + m2] w_P1^{m1 k1} ].
//
// Column pass: for each m2, the P1-point FFT over m1 (pruned: only the first
// LZ1 values of m1 can be nonzero, so R1 = P1/LZ1 pre-twiddled LZ1-point
// FFTs replace it), times w_P^{m2 k1}, written to a workspace W[k1][m2].
// Row pass: the P2-point FFT of each row k1 gives Y[k1 + P1 k2] at row k1,
// column k2.  Each CTA handles a few columns (or rows) so that every global
// access touches runs of consecutive elements.
//
// Padded FFT (P = H = N_FFT/2 after packing sample pairs): the row pass
// transforms row k1 together with its mirror row P1 - k1, which holds the
// partners Z[H - k] the real-input unpack needs, and writes X directly.
//
// Bluestein: the row pass runs the forward row FFT, the product with FFT(v)
// (stored in the same [k1][k2] order), and the inverse row FFT, then applies
// w_L^{-k1 n2}; an inverse column pass finishes the inverse FFT
// (n = n2 + P2 n1) and stores only the M outputs with the post-chirp.
//
// The twiddles w_P^i come from two small float64-generated tables,
// w_P^i = hi[i >> S] lo[i & (2^S - 1)].
#include "fft_block.cuh"
#include "spec_internal.h"

namespace spec {

constexpr int kRow = 512;            // P2: points per row
constexpr int kRowsPerCta = 8;       // rows per CTA in the row passes (and mirror rows for the real FFT)
// Row stride in the real row pass: odd in 8-byte words, so that the unpack's
// reads of the same column in 16 rows fall in different banks.
constexpr int kRowStride = kRow + kRow / 16 + 1;

struct Tw2 {
    const float2* hi;
    const float2* lo;
    int S;                           // lo holds 2^S entries
    int logP;                        // table period P = 2^logP
};

// e^{-j 2 pi i / 2^logP}
__device__ __forceinline__ float2 tw2(const Tw2& w, uint32_t i) {
    i &= (1u << w.logP) - 1u;
    return cmul(__ldg(w.hi + (i >> w.S)), __ldg(w.lo + (i & ((1u << w.S) - 1u))));
}

int tw2_split(int logP) { return (logP + 1) / 2; }
int tw2_entries(int logP) { return (1 << (logP - tw2_split(logP))) + (1 << tw2_split(logP)); }

void tw2_fill(int logP, float2* host) {
    const double two_pi = 6.283185307179586476925286766559;
    const int S = tw2_split(logP);
    const int64_t P = int64_t(1) << logP;
    auto w = [&](int64_t i) {
        const double ang = two_pi * (double)(i % P) / (double)P;
        return make_float2((float)std::cos(ang), (float)-std::sin(ang));
    };
    float2* o = host;
    for (int64_t i = 0; i < (P >> S); ++i) *o++ = w(i << S);
    for (int64_t i = 0; i < (int64_t(1) << S); ++i) *o++ = w(i);
}

static Tw2 tw2_view(const float2* tab, int logP) {
    Tw2 t;
    t.S = tw2_split(logP);
    t.logP = logP;
    t.hi = tab;
    t.lo = tab + (1 << (logP - t.S));
    return t;
}

// Shared-memory stride between the column FFTs of a CTA.  A warp holds the
// same element of 32 different columns, so the stride is made 1 modulo 16
// (in 8-byte words): the warp's accesses then spread over all banks.
__host__ __device__ constexpr int col_stride(int LF) {
    return padded_len(LF) + (17 - padded_len(LF) % 16) % 16;
}

// ------------------------------------------------------------ column pass --
enum ColInput : int {
    kPairs = 0,      // z[m] = x[2m] + j x[2m+1] (padded real FFT)
    kChirped = 1,    // x[m] pre[m] (Bluestein pre-multiply)
    kKernel = 2,     // the wrapped chirp kernel v[m] / L (table build)
};

struct ColArgs {
    int input;
    const float* x;
    int64_t ld_x;
    int n;                           // real samples (kPairs, kChirped)
    const float2* pre;               // kChirped
    int nk, mk;                      // kKernel: v nonzero for m < mk and m > P - nk
    uint64_t Bh;                     // kKernel: v[m] = e^{+j 2 pi Bh m^2}
    float scale;                     // kKernel
    int64_t batch;
    int logP, logP1, logR1;          // P = P1 P2; R1 = P1 / LZ1
    int G;                           // columns per CTA
    Tw2 tw;                          // period 2^tw.logP >= P
    const float2* btw;               // BlockFFT<LZ1> twiddles
    float2* W;                       // [batch][P1][P2]
};

// Two CTAs per SM up to 1024-point columns: at 64 registers the 512- and
// 1024-point forms spill ~150 bytes, yet the passes wait mostly on global
// loads and twice the warps hide more of it (measured on a 2^19-point
// Bluestein of 256 traces: 2.37 ms per call at one CTA per SM, 1.88 ms with
// this pass and the inverse column pass at two).
template <int LZ1>
__global__ void __launch_bounds__(512, LZ1 >= 2048 ? 1 : 2) k_long_cols(ColArgs a) {
    using FFT = BlockFFT<LZ1, false>;
    constexpr int E = FFT::E, T = FFT::T;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % a.G;                 // column within the group
    const int t = threadIdx.x / a.G;                 // thread within the column FFT
    const int groups = kRow / a.G;
    const int m2 = (blockIdx.x % groups) * a.G + c;
    const int r = blockIdx.x / groups;               // residue
    const int64_t b = blockIdx.y;
    const int P1 = 1 << a.logP1;
    const int up = a.tw.logP - a.logP;               // table index scale for w_P
    const int up1 = a.tw.logP - a.logP1;             // ... and for w_P1
    float2* s = smem + c * col_stride(LZ1);

    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int m1 = t + T * i;
        const int64_t m = (int64_t)kRow * m1 + m2;
        float2 y = make_float2(0.f, 0.f);
        if (a.input == kPairs) {
            const float* xr = a.x + b * a.ld_x;
            if (2 * m < a.n) y.x = __ldg(xr + 2 * m);
            if (2 * m + 1 < a.n) y.y = __ldg(xr + 2 * m + 1);
        } else if (a.input == kChirped) {
            if (m < a.n) y = cscale(__ldg(a.pre + m), __ldg(a.x + b * a.ld_x + m));
        } else {
            const int64_t P = int64_t(1) << a.logP;
            int64_t mm = 0;
            bool nz = true;
            if (m < a.mk) mm = m;
            else if (m > P - a.nk) mm = m - P;
            else nz = false;
            if (nz) {
                // e^{+j 2 pi Bh mm^2}: exact phase reduction in 64-bit fixed point
                y = cscale(unit_fixed_f64(a.Bh * (uint64_t)(mm * mm), false), a.scale);
            }
        }
        // residue pre-twiddle w_P1^{r m1}
        if (r != 0) y = cmul(y, tw2(a.tw, (uint32_t)(((int64_t)r * m1) & (P1 - 1)) << up1));
        v[i] = y;
    }
    FFT::run(v, s, t, a.btw);
    float2* Wb = a.W + (b << a.logP);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int k1 = ((t + T * i) << a.logR1) + r;
        const uint32_t idx = (uint32_t)(((int64_t)m2 * k1) & ((int64_t(1) << a.logP) - 1));
        Wb[(int64_t)k1 * kRow + m2] = cmul(v[i], tw2(a.tw, idx << up));
    }
}

// --------------------------------------------- row pass, padded real FFT --
struct RowRealArgs {
    int64_t batch;
    int logP1;                       // P1 rows
    int logH;                        // H = P1 P2
    const float2* W;
    float2* X;
    int64_t ld_X;
    Tw2 tw;                          // period 2H (the unpack twiddle e^{-j 2 pi k / N_FFT})
    const float2* btw;               // BlockFFT<kRow> twiddles
};

__global__ void __launch_bounds__(2 * kRowsPerCta * kRow / 16, 2) k_long_rows_real(RowRealArgs a) {
    using FFT = BlockFFT<kRow, false>;
    constexpr int E = FFT::E, T = FFT::T;
    constexpr int G = kRowsPerCta;
    extern __shared__ float2 smem[];
    const int P1 = 1 << a.logP1;
    const int H = 1 << a.logH;
    const int j = blockIdx.x;
    const int64_t b = blockIdx.y;
    const int slot = threadIdx.x / T;                // 0 .. 2G-1
    const int t = threadIdx.x % T;
    auto row_of = [&](int sl) {
        const int i = sl % G;
        if (sl < G) return j * G + i;
        if (j == 0 && i == 0) return P1 / 2;         // row 0 is its own mirror; take the self-mirrored P1/2
        return P1 - j * G - i;
    };
    const int row = row_of(slot);
    float2* s = smem + slot * kRowStride;
    const float2* Wr = a.W + (b << a.logH) + (int64_t)row * kRow;
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = __ldg(Wr + t + T * i);
    FFT::run(v, s, t, a.btw);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < E; ++i) s[pidx(t + T * i)] = v[i];     // Z[row + P1 k2] at k2
    __syncthreads();

    // unpack: X[k] = (A + conj B)/2 - j/2 w^k (A - conj B), A = Z[k], B = Z[H - k]
    float2* Xb = a.X + b * a.ld_X;
    const int total = 2 * G * kRow;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int ii = e % G;
        const int blk = (e / G) & 1;
        const int k2 = e / (2 * G);
        const int sl = blk * G + ii;
        const int rw = row_of(sl);
        int psl, pk2;
        if (rw == 0) { psl = sl; pk2 = (kRow - k2) & (kRow - 1); }
        else if (rw == P1 / 2) { psl = sl; pk2 = kRow - 1 - k2; }
        else { psl = sl < G ? sl + G : sl - G; pk2 = kRow - 1 - k2; }
        const float2 A = smem[sl * kRowStride + pidx(k2)];
        const float2 B = smem[psl * kRowStride + pidx(pk2)];
        const int k = rw + P1 * k2;
        const float2 w = tw2(a.tw, (uint32_t)k);
        const float2 sp = mul2(make_float2(A.x + B.x, A.y - B.y), make_float2(0.5f, 0.5f));
        const float2 dm = mul2(make_float2(A.x - B.x, A.y + B.y), make_float2(0.5f, 0.5f));
        const float2 wd = cmul(w, dm);
        Xb[k] = make_float2(sp.x + wd.y, sp.y - wd.x);
        if (k == 0) {
            // X[H] = sum x[even] - sum x[odd] = Re Z[0] - Im Z[0]
            Xb[H] = make_float2(A.x - A.y, 0.f);
        }
    }
}

// ------------------------------------- row pass, complex (Bluestein, V) --
struct RowC2cArgs {
    int64_t batch;
    int logP;                        // P = P1 P2 (the rows are P1 = P / kRow)
    float2* W;                       // [batch][P1][P2], transformed in place
    const float2* Vp;                // conv: FFT(v)/L in the same [k1][k2] order
    Tw2 tw;                          // period P
    const float2* btw;
};

// MODE 0: Bluestein row step (forward FFT, x V, inverse FFT, x w_P^{-k1 n2});
// MODE 1: forward row FFT only (builds V in [k1][k2] order).
template <int MODE>
__global__ void __launch_bounds__(kRowsPerCta * kRow / 16, 4) k_long_rows_c2c(RowC2cArgs a) {
    using Fw = BlockFFT<kRow, false>;
    using Iv = BlockFFT<kRow, true>;
    constexpr int E = Fw::E, T = Fw::T;
    extern __shared__ float2 smem[];
    const int slot = threadIdx.x / T;
    const int t = threadIdx.x % T;
    const int k1 = blockIdx.x * kRowsPerCta + slot;
    const int64_t b = blockIdx.y;
    float2* s = smem + slot * padded_len(kRow);
    float2* Wr = a.W + (b << a.logP) + (int64_t)k1 * kRow;
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = Wr[t + T * i];
    Fw::run(v, s, t, a.btw);
    if (MODE == 0) {
        const float2* Vr = a.Vp + (int64_t)k1 * kRow;
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = cmul(v[i], __ldg(Vr + t + T * i));
        int ti = t;                  // opaque copy: keeps the two FFTs' index math apart (register pressure)
        asm volatile("" : "+r"(ti));
        Iv::run(v, s, ti, a.btw);
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int n2 = t + T * i;
            const uint32_t idx = (uint32_t)(((int64_t)k1 * n2) & ((int64_t(1) << a.logP) - 1));
            v[i] = cmulc(v[i], tw2(a.tw, idx));                       // x w_P^{-k1 n2}
        }
    }
#pragma unroll
    for (int i = 0; i < E; ++i) Wr[t + T * i] = v[i];
}

// ------------------------------ inverse column pass with the post-chirp --
struct ColInvArgs {
    int64_t batch;
    int logP;
    int m;                           // outputs kept: n < m
    int G;
    const float2* W;                 // [batch][P1][P2] after the row step
    const float2* post;              // e^{-j 2 pi Bh k^2}, k < m
    float2* X;
    int64_t ld_X;
    const float2* btw;               // BlockFFT<P1> twiddles
};

template <int P1>
__global__ void __launch_bounds__(512, P1 >= 2048 ? 1 : 2) k_long_cols_inv(ColInvArgs a) {
    using Iv = BlockFFT<P1, true>;
    constexpr int E = Iv::E, T = Iv::T;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % a.G;
    const int t = threadIdx.x / a.G;
    const int n2 = blockIdx.x * a.G + c;
    const int64_t b = blockIdx.y;
    float2* s = smem + c * col_stride(P1);
    const float2* Wb = a.W + (b << a.logP);
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = __ldg(Wb + (int64_t)(t + T * i) * kRow + n2);
    Iv::run(v, s, t, a.btw);
    float2* Xb = a.X + b * a.ld_X;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int64_t nn = (int64_t)kRow * (t + T * i) + n2;
        if (nn < a.m) Xb[nn] = cmul(v[i], __ldg(a.post + nn));
    }
}

// ------------------------------------------------------------ dispatch ----
using ColKernel = void (*)(ColArgs);
using ColInvKernel = void (*)(ColInvArgs);

static ColKernel col_kernel_for(int LZ1) {
    switch (LZ1) {
        case 16: return k_long_cols<16>;
        case 32: return k_long_cols<32>;
        case 64: return k_long_cols<64>;
        case 128: return k_long_cols<128>;
        case 256: return k_long_cols<256>;
        case 512: return k_long_cols<512>;
        case 1024: return k_long_cols<1024>;
        case 2048: return k_long_cols<2048>;
        case 4096: return k_long_cols<4096>;
        case 8192: return k_long_cols<8192>;
        default: return nullptr;
    }
}

static ColInvKernel colinv_kernel_for(int P1) {
    switch (P1) {
        case 32: return k_long_cols_inv<32>;
        case 64: return k_long_cols_inv<64>;
        case 128: return k_long_cols_inv<128>;
        case 256: return k_long_cols_inv<256>;
        case 512: return k_long_cols_inv<512>;
        case 1024: return k_long_cols_inv<1024>;
        case 2048: return k_long_cols_inv<2048>;
        case 4096: return k_long_cols_inv<4096>;
        case 8192: return k_long_cols_inv<8192>;
        default: return nullptr;
    }
}

// Columns per CTA of a column pass over LF-point column FFTs: as many as fit
// in 512 threads and 8192 staged points, at most 32 (256-byte runs).
static int cols_per_cta(int LF) { return std::max(1, std::min(32, kTile / LF)); }

static cudaError_t set_smem(const void* k, size_t smem) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

static cudaError_t launch_cols(const LongPlan& p, ColArgs a, int64_t batch, cudaStream_t st) {
    ColKernel k = col_kernel_for(p.LZ1);
    if (!k) return cudaErrorInvalidValue;
    const int G = cols_per_cta(p.LZ1);
    a.G = G;
    const size_t smem = (size_t)G * col_stride(p.LZ1) * sizeof(float2);
    cudaError_t e = set_smem((const void*)k, smem);
    if (e != cudaSuccess) return e;
    const int T = std::max(1, p.LZ1 / 16);
    dim3 grid((unsigned)((kRow / G) << p.logR1), (unsigned)batch);
    k<<<grid, G * T, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- plans ---
bool long_fft_plan(int64_t n, int64_t n_fft, LongPlan* p, std::string* why) {
    *p = LongPlan();
    const int64_t H = n_fft / 2;
    const int64_t P1 = H / kRow;
    if (H < (int64_t)kRow * 2 * kRowsPerCta || P1 > (int64_t(1) << 16)) {
        *why = "multi-pass FFT: n_fft must be in [8192, 2^26]";
        return false;
    }
    const int64_t nz = (n + 1) / 2;                              // packed complex samples
    int64_t LZ1 = next_pow2((nz + kRow - 1) / kRow);
    LZ1 = std::min<int64_t>(std::max<int64_t>(LZ1, 16), P1);
    if (LZ1 > kTile) {
        *why = "multi-pass FFT: more than 8192 x 1024 samples per trace";
        return false;
    }
    p->logP = ilog2(H);
    p->logP1 = ilog2(P1);
    p->LZ1 = (int)LZ1;
    p->logR1 = ilog2(P1 / LZ1);
    p->logTw = p->logP + 1;                                      // table over N_FFT = 2H
    p->work_per_trace = H;
    return true;
}

bool long_czt_plan(int64_t n, int64_t m, LongPlan* p, std::string* why) {
    *p = LongPlan();
    const int64_t L = std::max<int64_t>(next_pow2(n + m - 1), (int64_t)kRow * 64);
    const int64_t P1 = L / kRow;
    if (P1 > kTile) {
        *why = "multi-pass CZT: N + M - 1 above 2^22";
        return false;
    }
    int64_t LZ1 = next_pow2((n + kRow - 1) / kRow);
    LZ1 = std::min<int64_t>(std::max<int64_t>(LZ1, 16), P1);
    p->logP = ilog2(L);
    p->logP1 = ilog2(P1);
    p->LZ1 = (int)LZ1;
    p->logR1 = ilog2(P1 / LZ1);
    p->logTw = p->logP;
    p->work_per_trace = L;
    return true;
}

// ------------------------------------------------------------- launches ---
cudaError_t long_fft_launch(const LongPlan& p, const float* x, int64_t batch, int n, int64_t ld_x,
                            const float2* block_tw_base, const float2* tw_tab, float2* work, int64_t work_traces,
                            float2* X, int64_t ld_X, cudaStream_t st) {
    const Tw2 tw = tw2_view(tw_tab, p.logTw);
    const int P1 = 1 << p.logP1;
    for (int64_t b0 = 0; b0 < batch; b0 += work_traces) {
        const int64_t nb = std::min(work_traces, batch - b0);
        ColArgs c = {};
        c.input = kPairs;
        c.x = x + b0 * ld_x; c.ld_x = ld_x; c.n = n;
        c.batch = nb;
        c.logP = p.logP; c.logP1 = p.logP1; c.logR1 = p.logR1;
        c.tw = tw;
        c.btw = block_tw_base + block_twiddle_offset(p.LZ1);
        c.W = work;
        cudaError_t e = launch_cols(p, c, nb, st);
        if (e != cudaSuccess) return e;
        RowRealArgs r = {};
        r.batch = nb; r.logP1 = p.logP1; r.logH = p.logP;
        r.W = work; r.X = X + b0 * ld_X; r.ld_X = ld_X;
        r.tw = tw;
        r.btw = block_tw_base + block_twiddle_offset(kRow);
        const size_t smem = (size_t)2 * kRowsPerCta * kRowStride * sizeof(float2);
        e = set_smem((const void*)k_long_rows_real, smem);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)(P1 / (2 * kRowsPerCta)), (unsigned)nb);
        k_long_rows_real<<<grid, 2 * kRowsPerCta * (kRow / 16), smem, st>>>(r);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t launch_rows_c2c(int mode, int logP, float2* W, const float2* Vp, const Tw2& tw,
                                   const float2* btw, int64_t nb, cudaStream_t st) {
    RowC2cArgs r = {};
    r.batch = nb; r.logP = logP; r.W = W; r.Vp = Vp; r.tw = tw; r.btw = btw;
    const size_t smem = (size_t)kRowsPerCta * padded_len(kRow) * sizeof(float2);
    auto k = mode == 0 ? k_long_rows_c2c<0> : k_long_rows_c2c<1>;
    cudaError_t e = set_smem((const void*)k, smem);
    if (e != cudaSuccess) return e;
    const int P1 = (1 << logP) / kRow;
    dim3 grid((unsigned)(P1 / kRowsPerCta), (unsigned)nb);
    k<<<grid, kRowsPerCta * (kRow / 16), smem, st>>>(r);
    return cudaGetLastError();
}

int long_czt_table_entries(const LongPlan& p) { return tw2_entries(p.logTw); }

cudaError_t long_czt_build_tables(const LongPlan& p, const CztTables& t, const float2* block_tw_base,
                                  float2* tw_tab, cudaStream_t st) {
    cudaError_t e = czt_pre_post_launch(t, st);
    if (e != cudaSuccess) return e;
    const Tw2 tw = tw2_view(tw_tab, p.logTw);
    // V = FFT_L(v)/L, dense (no pruning), written in [k1][k2] order
    LongPlan q = p;
    q.LZ1 = 1 << p.logP1;
    q.logR1 = 0;
    ColArgs c = {};
    c.input = kKernel;
    c.nk = t.n; c.mk = t.m; c.Bh = t.Bh;
    c.scale = 1.0f / (float)(int64_t(1) << p.logP);
    c.batch = 1;
    c.logP = p.logP; c.logP1 = p.logP1; c.logR1 = 0;
    c.tw = tw;
    c.btw = block_tw_base + block_twiddle_offset(q.LZ1);
    c.W = t.V;
    e = launch_cols(q, c, 1, st);
    if (e != cudaSuccess) return e;
    return launch_rows_c2c(1, p.logP, t.V, nullptr, tw, block_tw_base + block_twiddle_offset(kRow), 1, st);
}

cudaError_t long_czt_launch(const LongPlan& p, const CztTables& t, const float2* tw_tab, const float* x,
                            int64_t batch, int64_t ld_x, const float2* block_tw_base, float2* work,
                            int64_t work_traces, float2* X, int64_t ld_X, cudaStream_t st) {
    const Tw2 tw = tw2_view(tw_tab, p.logTw);
    const int P1 = 1 << p.logP1;
    ColInvKernel ki = colinv_kernel_for(P1);
    if (!ki) return cudaErrorInvalidValue;
    const int Gi = cols_per_cta(P1);
    const size_t smem_i = (size_t)Gi * col_stride(P1) * sizeof(float2);
    cudaError_t e = set_smem((const void*)ki, smem_i);
    if (e != cudaSuccess) return e;
    const int live_cols = (int)std::min<int64_t>(kRow, t.m);
    for (int64_t b0 = 0; b0 < batch; b0 += work_traces) {
        const int64_t nb = std::min(work_traces, batch - b0);
        ColArgs c = {};
        c.input = kChirped;
        c.x = x + b0 * ld_x; c.ld_x = ld_x; c.n = t.n; c.pre = t.pre;
        c.batch = nb;
        c.logP = p.logP; c.logP1 = p.logP1; c.logR1 = p.logR1;
        c.tw = tw;
        c.btw = block_tw_base + block_twiddle_offset(p.LZ1);
        c.W = work;
        e = launch_cols(p, c, nb, st);
        if (e != cudaSuccess) return e;
        e = launch_rows_c2c(0, p.logP, work, t.V, tw, block_tw_base + block_twiddle_offset(kRow), nb, st);
        if (e != cudaSuccess) return e;
        ColInvArgs ia = {};
        ia.batch = nb; ia.logP = p.logP; ia.m = t.m; ia.G = Gi;
        ia.W = work; ia.post = t.post; ia.X = X + b0 * ld_X; ia.ld_X = ld_X;
        ia.btw = block_tw_base + block_twiddle_offset(P1);
        dim3 grid((unsigned)((live_cols + Gi - 1) / Gi), (unsigned)nb);
        ki<<<grid, Gi * (P1 / 16), smem_i, st>>>(ia);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int long_fft_table_entries(const LongPlan& p) { return tw2_entries(p.logTw); }
void long_fill_tw(const LongPlan& p, float2* host) { tw2_fill(p.logTw, host); }

}  // namespace spec
