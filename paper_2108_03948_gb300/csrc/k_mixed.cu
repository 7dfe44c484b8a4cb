// k_mixed.cu -- zero-padded FFT (Section 2.1, Eq. 2-3) for a padded length
// N_FFT that is not a power of two but has only the factors 2, 3, 5 and 7:
// the lengths of the resolution sweep of Section 4 (N_FFT = fs/Delta f from
// Eq. 3, e.g. 500, 1000, 2000, 10000, 20000 = 2^k 5^j).
//
// The method is the padded FFT's (k_fft.cu) with a mixed-radix engine:
//  1. pack sample pairs, z[m] = x[2m] + j x[2m+1], H = N_FFT/2 complex points
//     of which the first ceil(N/2) can be nonzero;
//  2. prune the padding: with H = R LZ (LZ a divisor of H at least
//     ceil(N/2)), bin R q + r of the H-point DFT is bin q of the LZ-point DFT
//     of z[m] w_H^{r m}, so R LZ-point DFTs replace the H-point one;
//  3. each LZ-point DFT runs as Stockham passes of radix 8, 4, 2, 3, 5 or 7
//     (the factors of LZ), all R of them at once, through two shared-memory
//     buffers of H values;
//  4. unpack X[k] = (Z[k] + conj Z[H-k])/2 - j/2 w^k (Z[k] - conj Z[H-k]),
//     w = e^{-j 2 pi/N_FFT}, coalesced stores.
// F traces per CTA (a power-of-two number of threads per trace, about H/4,
// each trace on its own named barrier); the pre-twiddles, pass twiddles and
// unpack twiddles come from one float64-generated table per plan, the roots
// of the odd radices are constants, and every index split (residue and
// position, butterfly and twiddle index) is a float-reciprocal division with
// one correction step instead of an integer division.
#include "fft_block.cuh"
#include "spec_internal.h"

namespace spec {

namespace {

constexpr int kMixedCta = 1024;       // threads per CTA at most (F traces of TT threads)

// X[k] and X[H - k] from A = Z[k], B = Z[H - k] (the real-input unpack)
__device__ __forceinline__ void unpack_pair_mixed(float2* Xr, int k, int H, float2 A, float2 B, float2 w) {
    const float2 sp = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
    const float2 dm = make_float2(0.5f * (A.x - B.x), 0.5f * (A.y + B.y));
    const float2 wd = cmul(w, dm);
    Xr[k] = make_float2(sp.x + wd.y, sp.y - wd.x);
    if (H - k != k) Xr[H - k] = make_float2(sp.x - wd.y, -sp.y - wd.x);
}

// q = x / d, x - q d for 0 <= x < 2^24 without an integer division: the
// float quotient (reciprocal rounded, so off by at most one) and one
// correction step
__device__ __forceinline__ int fdivmod(int x, int d, float rcp, int* rem) {
    int q = __float2int_rz((float)x * rcp);
    int r = x - q * d;
    if (r < 0) { --q; r += d; }
    else if (r >= d) { ++q; r -= d; }
    *rem = r;
    return q;
}

struct MixedArgs {
    const float* x;
    int64_t batch;
    int n;
    int64_t ld_x;
    float2* X;
    int64_t ld_X;
    int H, LZ, R, npass, TT, F;
    float rLZ, rR;
    int radix[kMixedMaxPasses], per[kMixedMaxPasses], ns[kMixedMaxPasses], twoff[kMixedMaxPasses];
    float rper[kMixedMaxPasses], rns[kMixedMaxPasses];
    const float2* tab;         // MixedPlan layout: pre-twiddles | pass twiddles | unpack
    int pre_off, unpack_off;
};

// cos and sin of 2 pi m / r, m < r, for the odd radices
template <int r>
__device__ __forceinline__ float root_c(int m) {
    if constexpr (r == 3) return m == 0 ? 1.f : -0.5f;
    else if constexpr (r == 5)
        return m == 0 ? 1.f : (m == 1 || m == 4) ? 0.30901699437494745f : -0.8090169943749475f;
    else
        return m == 0 ? 1.f : (m == 1 || m == 6) ? 0.6234898018587336f
                            : (m == 2 || m == 5) ? -0.22252093395631440f : -0.9009688679024191f;
}
template <int r>
__device__ __forceinline__ float root_s(int m) {
    if constexpr (r == 3) return m == 0 ? 0.f : m == 1 ? 0.8660254037844386f : -0.8660254037844386f;
    else if constexpr (r == 5)
        return m == 0 ? 0.f : m == 1 ? 0.9510565162951535f : m == 2 ? 0.5877852522924731f
                            : m == 3 ? -0.5877852522924731f : -0.9510565162951535f;
    else
        return m == 0 ? 0.f : m == 1 ? 0.7818314824680298f : m == 2 ? 0.9749279121818236f
                            : m == 3 ? 0.4338837391175581f : m == 4 ? -0.4338837391175581f
                            : m == 5 ? -0.9749279121818236f : -0.7818314824680298f;
}

// y = DFT_r(v) (forward) for an odd radix, from the pair sums and
// differences: X[k] = v0 + sum_i s_i cos(2 pi i k/r) - j sum_i d_i sin(2 pi i k/r),
// s_i = v_i + v_{r-i}, d_i = v_i - v_{r-i}, and X[r-k] with the sine part negated
template <int r>
__device__ __forceinline__ void dft_odd(float2 (&v)[8]) {
    constexpr int h = (r - 1) / 2;
    float2 sm[h], df[h];
#pragma unroll
    for (int i = 1; i <= h; ++i) {
        sm[i - 1] = cadd(v[i], v[r - i]);
        df[i - 1] = csub(v[i], v[r - i]);
    }
    float2 y[r];
    y[0] = v[0];
#pragma unroll
    for (int i = 0; i < h; ++i) y[0] = cadd(y[0], sm[i]);
#pragma unroll
    for (int k = 1; k <= h; ++k) {
        float2 c = v[0], sj = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 1; i <= h; ++i) {
            const float cc = root_c<r>((i * k) % r), ss = root_s<r>((i * k) % r);
            c = make_float2(fmaf(cc, sm[i - 1].x, c.x), fmaf(cc, sm[i - 1].y, c.y));
            sj = make_float2(fmaf(ss, df[i - 1].x, sj.x), fmaf(ss, df[i - 1].y, sj.y));
        }
        // -j sj = (sj.y, -sj.x)
        y[k] = make_float2(c.x + sj.y, c.y - sj.x);
        y[r - k] = make_float2(c.x - sj.y, c.y + sj.x);
    }
#pragma unroll
    for (int k = 0; k < r; ++k) v[k] = y[k];
}

__device__ __forceinline__ void dft_any(int r, float2 (&v)[8]) {
    switch (r) {
        case 2: dft2<false>(v[0], v[1]); break;
        case 4: dft4<false>(v[0], v[1], v[2], v[3]); break;
        case 8: dft8<false>(v); break;
        case 3: dft_odd<3>(v); break;
        case 5: dft_odd<5>(v); break;
        default: dft_odd<7>(v); break;
    }
}

__global__ void __launch_bounds__(kMixedCta) k_fft_mixed(MixedArgs a) {
    extern __shared__ float2 smem[];
    const int H = a.H, LZ = a.LZ, TT = a.TT;
    const int f = threadIdx.x / TT;
    const int tid = threadIdx.x - f * TT;
    const int64_t b = (int64_t)blockIdx.x * a.F + f;
    const bool live = b < a.batch;
    // the F traces of a CTA synchronise on their own named barriers
    const int bar = a.F > 1 ? 1 + f : 0;
    float2* src = smem + (size_t)f * 2 * H;
    float2* dst = src + H;
    const float* xr = a.x + (live ? b : 0) * a.ld_x;
    const int n = a.n;
    // 1-2. packed, pre-twiddled input of every residue: src[r LZ + m]
    for (int idx = tid; idx < H; idx += TT) {
        int m;
        fdivmod(idx, LZ, a.rLZ, &m);
        const float re = live && 2 * m < n ? __ldg(xr + 2 * m) : 0.f;
        const float im = live && 2 * m + 1 < n ? __ldg(xr + 2 * m + 1) : 0.f;
        src[idx] = cmul(make_float2(re, im), __ldg(a.tab + a.pre_off + idx));
    }
    group_sync(bar, TT);
    // 3. Stockham passes over all R residue DFTs at once
    for (int p = 0; p < a.npass; ++p) {
        const int r = a.radix[p], per = a.per[p], NS = a.ns[p];
        const float rper = a.rper[p], rns = a.rns[p];
        const float2* tw = a.tab + a.twoff[p];
        for (int bi = tid; bi < H / r; bi += TT) {
            int j, k;
            const int res = fdivmod(bi, per, rper, &j);
            const int jk = fdivmod(j, NS, rns, &k);
            const float2* in = src + res * LZ + j;
            float2 v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < r) v[i] = in[i * per];
            if (NS > 1) {
#pragma unroll
                for (int i = 1; i < 8; ++i)
                    if (i < r) v[i] = cmul(v[i], __ldg(tw + (i - 1) * NS + k));
            }
            dft_any(r, v);
            float2* out = dst + res * LZ + jk * NS * r + k;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < r) out[i * NS] = v[i];
        }
        group_sync(bar, TT);
        float2* t = src;
        src = dst;
        dst = t;
    }
    if (!live) return;
    // 4. unpack the pairs (k, H - k); Z[k] = src[(k mod R) LZ + k / R]
    float2* Xr = a.X + b * a.ld_X;
    const float2* wk = a.tab + a.unpack_off;
    for (int k = tid; k <= H / 2; k += TT) {
        const int km = k == 0 ? 0 : H - k;
        int ra, rb;
        const int qa = fdivmod(k, a.R, a.rR, &ra);
        const int qb = fdivmod(km, a.R, a.rR, &rb);
        unpack_pair_mixed(Xr, k, H, src[ra * LZ + qa], src[rb * LZ + qb], __ldg(wk + k));
    }
}

// ---------------------------------------------------------------------------
// Register-resident form for residue lengths 250, 500 and 1000 (LZ = 10 x
// 5 x 5, 10 x 10 x 5, 10 x 10 x 10: the residue DFTs of the paper's N = 500
// traces and of 1000 / 2000-sample ones).  Each residue DFT runs on T = LZ/10
// threads holding 10 elements each in registers (t + T i before and after
// the transform, as BlockFFT does for powers of two): Stockham passes of
// radix 10 (two radix-5 DFTs and a radix-2 combination) and 5, each followed
// by one exchange through the residue's shared-memory area, with the pass
// twiddles from the plan's table.  Residues are padded to LZ + 1 values, so
// the unpack's reads of Z[k] for consecutive k (consecutive residues) fall on
// different banks.
template <int LZ> struct MixedRegShape;
template <> struct MixedRegShape<250> {
    static constexpr int rad(int p) { return p == 0 ? 10 : 5; }
};
template <> struct MixedRegShape<500> {
    static constexpr int rad(int p) { return p < 2 ? 10 : 5; }
};
template <> struct MixedRegShape<1000> {
    static constexpr int rad(int p) { return 10; }
};

template <int LZ> __host__ __device__ constexpr int mreg_ns(int p) {
    return p == 0 ? 1 : mreg_ns<LZ>(p - 1) * MixedRegShape<LZ>::rad(p - 1);
}
// offset of pass p's twiddles in the plan's pass table (passes with NS > 1)
template <int LZ> __host__ __device__ constexpr int mreg_twoff(int p) {
    return p <= 1 ? 0 : mreg_twoff<LZ>(p - 1) + (MixedRegShape<LZ>::rad(p - 1) - 1) * mreg_ns<LZ>(p - 1);
}

__device__ __forceinline__ void dft5(float2* v) {
    float2 w[8] = {v[0], v[1], v[2], v[3], v[4]};
    dft_odd<5>(w);
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = w[i];
}

// 10 = 2 x 5: X[k] = E[k] + w10^k O[k], X[k + 5] = E[k] - w10^k O[k]
__device__ __forceinline__ void dft10(float2 (&v)[10]) {
    float2 e[5] = {v[0], v[2], v[4], v[6], v[8]};
    float2 o[5] = {v[1], v[3], v[5], v[7], v[9]};
    dft5(e);
    dft5(o);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        // w10^k = e^{-j pi k/5} = e^{-j pi (32 k/5)/32}: cos(pi k/5), -sin(pi k/5)
        const float c = k == 0 ? 1.f : k == 1 ? 0.80901699437494742f : k == 2 ? 0.30901699437494742f
                      : k == 3 ? -0.30901699437494742f : -0.80901699437494742f;
        const float sn = k == 0 ? 0.f : (k == 1 || k == 4) ? 0.58778525229247313f : 0.95105651629515357f;
        const float2 t = make_float2(fmaf(o[k].x, c, o[k].y * sn), fmaf(o[k].y, c, -o[k].x * sn));
        v[k] = cadd(e[k], t);
        v[k + 5] = csub(e[k], t);
    }
}

template <int LZ, int P>
__device__ __forceinline__ void mreg_compute(float2 (&v)[10], int t, const float2* tw) {
    constexpr int T = LZ / 10;
    constexpr int RP = MixedRegShape<LZ>::rad(P);
    constexpr int NS = mreg_ns<LZ>(P);
    constexpr int NB = 10 / RP;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        float2 u[10];
#pragma unroll
        for (int r = 0; r < RP; ++r) u[r] = v[b + r * NB];
        if constexpr (NS > 1) {
            const int k = (t + T * b) % NS;
            const float2* twp = tw + mreg_twoff<LZ>(P) + k;
#pragma unroll
            for (int r = 1; r < RP; ++r) u[r] = cmul(u[r], __ldg(twp + (r - 1) * NS));
        }
        if constexpr (RP == 10) dft10(u);
        else dft5(u);
#pragma unroll
        for (int r = 0; r < RP; ++r) v[b + r * NB] = u[r];
    }
}

// the outputs of pass P to their Stockham positions, then the thread's next
// inputs t + T i
template <int LZ, int P>
__device__ __forceinline__ void mreg_exchange(float2 (&v)[10], float2* s, int t) {
    constexpr int T = LZ / 10;
    constexpr int RP = MixedRegShape<LZ>::rad(P);
    constexpr int NS = mreg_ns<LZ>(P);
    constexpr int NB = 10 / RP;
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + T * b;
        const int k = j % NS;
        const int base = (j - k) * RP + k;
#pragma unroll
        for (int r = 0; r < RP; ++r) s[base + r * NS] = v[b + r * NB];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 10; ++i) v[i] = s[t + T * i];
}

struct MixedRegArgs {
    const float* x;
    int64_t batch;
    int n;
    int64_t ld_x;
    float2* X;
    int64_t ld_X;
    int H, R, F;
    float rR;
    const float2* tab;
    int pre_off, pass_off, unpack_off;
};

template <int LZ>
__global__ void __launch_bounds__(1000) k_fft_mixed_regs(MixedRegArgs a) {
    constexpr int E = 10, T = LZ / E, LZP = LZ + 1;
    static_assert(mreg_ns<LZ>(3) == LZ, "three passes of the shape cover LZ");
    extern __shared__ float2 smem[];
    const int R = a.R, H = a.H;
    const int PT = R * T;                            // threads per trace
    const int f = threadIdx.x / PT;
    const int lt = threadIdx.x - f * PT;
    const int res = lt / T;
    const int t = lt - res * T;
    const int64_t b = (int64_t)blockIdx.x * a.F + f;
    const bool live = b < a.batch;
    float2* zs = smem + (size_t)f * R * LZP;
    float2* s = zs + res * LZP;
    // 1-2. packed, pre-twiddled input of this thread's residue: m = t + T i
    float2 v[E];
    {
        const float* xr = a.x + (live ? b : 0) * a.ld_x;
        const float2* pre = a.tab + a.pre_off + res * LZ;
        const int n = a.n;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int m = t + T * i;
            const float re = live && 2 * m < n ? __ldg(xr + 2 * m) : 0.f;
            const float im = live && 2 * m + 1 < n ? __ldg(xr + 2 * m + 1) : 0.f;
            v[i] = cmul(make_float2(re, im), __ldg(pre + m));
        }
    }
    // 3. the residue DFT: three passes in registers
    const float2* tw = a.tab + a.pass_off;
    mreg_compute<LZ, 0>(v, t, tw);
    mreg_exchange<LZ, 0>(v, s, t);
    mreg_compute<LZ, 1>(v, t, tw);
    mreg_exchange<LZ, 1>(v, s, t);
    mreg_compute<LZ, 2>(v, t, tw);
    // Z[R q + res] at q = t + T i
    __syncthreads();
#pragma unroll
    for (int i = 0; i < E; ++i) s[t + T * i] = v[i];
    __syncthreads();
    if (!live) return;
    // 4. unpack the pairs (k, H - k); Z[k] = zs[(k mod R) LZP + k / R]
    float2* Xr = a.X + b * a.ld_X;
    const float2* wk = a.tab + a.unpack_off;
    for (int k = lt; k <= H / 2; k += PT) {
        const int km = k == 0 ? 0 : H - k;
        int ra, rb;
        const int qa = fdivmod(k, R, a.rR, &ra);
        const int qb = fdivmod(km, R, a.rR, &rb);
        unpack_pair_mixed(Xr, k, H, zs[ra * LZP + qa], zs[rb * LZP + qb], __ldg(wk + k));
    }
}

}  // namespace

// ------------------------------------------------------------------- host --

// Radices of an LZ-point DFT: powers of two as 8s (then one 4 or 2), then the
// odd factors; false if LZ has a prime factor above 7.
static bool mixed_radices(int LZ, std::vector<int>* out) {
    out->clear();
    int m = LZ;
    while (m % 8 == 0) { out->push_back(8); m /= 8; }
    if (m % 4 == 0) { out->push_back(4); m /= 4; }
    if (m % 2 == 0) { out->push_back(2); m /= 2; }
    for (int q : {3, 5, 7})
        while (m % q == 0) { out->push_back(q); m /= q; }
    return m == 1 && (int)out->size() <= kMixedMaxPasses;
}

bool mixed_plan(int64_t n, int64_t n_fft, MixedPlan* p, std::string* why) {
    *p = MixedPlan();
    if (n_fft % 2 != 0 || n_fft < 4) {
        *why = "mixed-radix FFT: N_FFT must be even";
        return false;
    }
    const int64_t H = n_fft / 2;
    if (H > kMixedMaxH) {
        *why = "mixed-radix FFT: N_FFT above the one-CTA size";
        return false;
    }
    const int64_t need = std::max<int64_t>(1, (n + 1) / 2);
    // the smallest divisor LZ of H with LZ >= ceil(N/2) whose factors are 2, 3, 5, 7
    std::vector<int> rad;
    for (int64_t LZ = need; LZ <= H; ++LZ) {
        if (H % LZ != 0) continue;
        if (!mixed_radices((int)LZ, &rad)) continue;
        p->H = (int)H;
        p->LZ = (int)LZ;
        p->R = (int)(H / LZ);
        p->radix = rad;
        // residue lengths with a register-resident kernel (one CTA of at most
        // 1000 threads per trace): its radix plan sets the table layout
        if ((LZ == 250 || LZ == 500 || LZ == 1000) && p->R * (LZ / 10) <= 1000) {
            p->regs = true;
            p->radix = LZ == 250 ? std::vector<int>{10, 5, 5}
                     : LZ == 500 ? std::vector<int>{10, 10, 5} : std::vector<int>{10, 10, 10};
        }
        rad = p->radix;
        // table: pre-twiddles [R][LZ] | pass twiddles | unpack
        int pass = 0, ns = 1;
        for (int r : rad) {
            if (ns > 1) pass += (r - 1) * ns;
            ns *= r;
        }
        p->pre_off = 0;
        p->pass_off = (int)H;
        p->root_off = p->pass_off + pass;
        p->unpack_off = p->root_off;
        p->entries = p->unpack_off + (int)(H / 2) + 1;
        p->smem = (size_t)2 * H * sizeof(float2);
        return true;
    }
    *why = "mixed-radix FFT: N_FFT/2 has a prime factor above 7";
    return false;
}

void mixed_fill_table(const MixedPlan& p, float2* host) {
    const double two_pi = 6.283185307179586476925286766559;
    auto w = [&](int64_t num, int64_t den) {     // e^{-j 2 pi num/den}, exact reduction
        const double ang = two_pi * (double)(num % den) / (double)den;
        return make_float2((float)std::cos(ang), (float)-std::sin(ang));
    };
    const int64_t H = p.H;
    for (int r = 0; r < p.R; ++r)
        for (int m = 0; m < p.LZ; ++m) host[p.pre_off + (int64_t)r * p.LZ + m] = w((int64_t)r * m, H);
    int off = p.pass_off, ns = 1;
    for (int r : p.radix) {
        if (ns > 1)
            for (int i = 1; i < r; ++i)
                for (int k = 0; k < ns; ++k) host[off + (i - 1) * ns + k] = w((int64_t)i * k, (int64_t)ns * r);
        if (ns > 1) off += (r - 1) * ns;
        ns *= r;
    }
    for (int64_t k = 0; k <= H / 2; ++k) host[p.unpack_off + k] = w(k, 2 * H);
}

static cudaError_t mixed_regs_launch(const MixedPlan& p, const float* x, int64_t batch, int n, int64_t ld_x,
                                     const float2* tab, float2* X, int64_t ld_X, cudaStream_t st) {
    MixedRegArgs a = {};
    a.x = x; a.batch = batch; a.n = n; a.ld_x = ld_x; a.X = X; a.ld_X = ld_X;
    a.H = p.H; a.R = p.R; a.rR = 1.0f / (float)p.R;
    a.tab = tab; a.pre_off = p.pre_off; a.pass_off = p.pass_off; a.unpack_off = p.unpack_off;
    const int PT = p.R * (p.LZ / 10);
    const size_t per = (size_t)p.R * (p.LZ + 1) * sizeof(float2);
    int F = std::max(1, 1000 / PT);
    while (F > 1 && (size_t)F * per > 100 * 1024) --F;
    a.F = F;
    const size_t smem = (size_t)F * per;
    const void* k = p.LZ == 250 ? (const void*)k_fft_mixed_regs<250>
                  : p.LZ == 500 ? (const void*)k_fft_mixed_regs<500> : (const void*)k_fft_mixed_regs<1000>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((batch + F - 1) / F);
    if (p.LZ == 250) k_fft_mixed_regs<250><<<grid, F * PT, smem, st>>>(a);
    else if (p.LZ == 500) k_fft_mixed_regs<500><<<grid, F * PT, smem, st>>>(a);
    else k_fft_mixed_regs<1000><<<grid, F * PT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t mixed_launch(const MixedPlan& p, const float* x, int64_t batch, int n, int64_t ld_x, const float2* tab,
                         float2* X, int64_t ld_X, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    if (p.regs) return mixed_regs_launch(p, x, batch, n, ld_x, tab, X, ld_X, st);
    MixedArgs a = {};
    a.x = x; a.batch = batch; a.n = n; a.ld_x = ld_x; a.X = X; a.ld_X = ld_X;
    a.H = p.H; a.LZ = p.LZ; a.R = p.R; a.npass = (int)p.radix.size();
    a.rLZ = 1.0f / (float)p.LZ;
    a.rR = 1.0f / (float)p.R;
    // threads per trace: about a quarter of H (a radix-4 pass in one sweep), a
    // power of two in [32, 1024]; short traces share a CTA of 256 threads (at
    // most 4 traces, one named barrier each)
    int TT = 32;
    while (TT < kMixedCta && TT < (p.H + 3) / 4) TT *= 2;
    a.TT = TT;
    a.F = std::max(1, std::min(4, 256 / TT));
    int ns = 1, off = p.pass_off;
    for (size_t i = 0; i < p.radix.size(); ++i) {
        const int r = p.radix[i];
        a.radix[i] = r;
        a.per[i] = p.LZ / r;
        a.ns[i] = ns;
        a.rper[i] = 1.0f / (float)a.per[i];
        a.rns[i] = 1.0f / (float)ns;
        a.twoff[i] = off;
        if (ns > 1) off += (r - 1) * ns;
        ns *= r;
    }
    a.tab = tab;
    a.pre_off = p.pre_off; a.unpack_off = p.unpack_off;
    const size_t smem = (size_t)a.F * 2 * p.H * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_fft_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fft_mixed<<<(unsigned)((batch + a.F - 1) / a.F), a.F * TT, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace spec
