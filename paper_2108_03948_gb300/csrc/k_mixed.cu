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
// One CTA per trace; every twiddle (pre-twiddles, pass twiddles, the roots of
// the odd radices, the unpack twiddle) comes from one float64-generated table
// per plan.
#include "fft_block.cuh"
#include "spec_internal.h"

namespace spec {

namespace {

constexpr int kMixedThreads = 512;

// X[k] and X[H - k] from A = Z[k], B = Z[H - k] (the real-input unpack)
__device__ __forceinline__ void unpack_pair_mixed(float2* Xr, int k, int H, float2 A, float2 B, float2 w) {
    const float2 sp = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
    const float2 dm = make_float2(0.5f * (A.x - B.x), 0.5f * (A.y + B.y));
    const float2 wd = cmul(w, dm);
    Xr[k] = make_float2(sp.x + wd.y, sp.y - wd.x);
    if (H - k != k) Xr[H - k] = make_float2(sp.x - wd.y, -sp.y - wd.x);
}

struct MixedArgs {
    const float* x;
    int64_t batch;
    int n;
    int64_t ld_x;
    float2* X;
    int64_t ld_X;
    int H, LZ, R, npass;
    int radix[kMixedMaxPasses];
    const float2* tab;         // MixedPlan layout (offsets below)
    int pre_off, pass_off, root_off, unpack_off;
};

// y = DFT_r(v) for an odd radix r (3, 5, 7) by its definition, with the
// r roots e^{-j 2 pi i/r} from the table (root[i], i < r)
template <int r>
__device__ __forceinline__ void dft_odd(float2 (&v)[8], const float2* root) {
    float2 w[r];
#pragma unroll
    for (int i = 0; i < r; ++i) w[i] = __ldg(root + i);
    float2 y[r];
#pragma unroll
    for (int k = 0; k < r; ++k) {
        float2 acc = v[0];
#pragma unroll
        for (int i = 1; i < r; ++i) acc = cadd(acc, cmul(v[i], w[(i * k) % r]));
        y[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < r; ++k) v[k] = y[k];
}

__device__ __forceinline__ void dft_any(int r, float2 (&v)[8], const float2* roots) {
    switch (r) {
        case 2: dft2<false>(v[0], v[1]); break;
        case 4: dft4<false>(v[0], v[1], v[2], v[3]); break;
        case 8: dft8<false>(v); break;
        case 3: dft_odd<3>(v, roots); break;
        case 5: dft_odd<5>(v, roots + 3); break;
        default: dft_odd<7>(v, roots + 8); break;
    }
}

__global__ void __launch_bounds__(kMixedThreads) k_fft_mixed(MixedArgs a) {
    extern __shared__ float2 smem[];
    const int H = a.H, LZ = a.LZ, R = a.R;
    float2* src = smem;
    float2* dst = smem + H;
    const int64_t b = blockIdx.x;
    const float* xr = a.x + b * a.ld_x;
    const int n = a.n;
    // 1-2. packed, pre-twiddled input of every residue: src[r LZ + m]
    for (int idx = threadIdx.x; idx < H; idx += kMixedThreads) {
        const int r = idx / LZ;
        const int m = idx - r * LZ;
        const float re = 2 * m < n ? __ldg(xr + 2 * m) : 0.f;
        const float im = 2 * m + 1 < n ? __ldg(xr + 2 * m + 1) : 0.f;
        src[idx] = cmul(make_float2(re, im), __ldg(a.tab + a.pre_off + idx));
    }
    __syncthreads();
    // 3. Stockham passes over all R residue DFTs at once
    const float2* roots = a.tab + a.root_off;
    int NS = 1, twoff = a.pass_off;
    for (int p = 0; p < a.npass; ++p) {
        const int r = a.radix[p];
        const int per = LZ / r;                 // butterflies per residue DFT
        for (int bi = threadIdx.x; bi < H / r; bi += kMixedThreads) {
            const int res = bi / per;
            const int j = bi - res * per;
            const int k = j % NS;
            const float2* in = src + res * LZ + j;
            float2 v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < r) v[i] = in[i * per];
            if (NS > 1) {
                const float2* tw = a.tab + twoff + k;
#pragma unroll
                for (int i = 1; i < 8; ++i)
                    if (i < r) v[i] = cmul(v[i], __ldg(tw + (i - 1) * NS));
            }
            dft_any(r, v, roots);
            float2* out = dst + res * LZ + (j - k) * r + k;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < r) out[i * NS] = v[i];
        }
        __syncthreads();
        float2* t = src;
        src = dst;
        dst = t;
        if (NS > 1) twoff += (r - 1) * NS;
        NS *= r;
    }
    // 4. unpack the pairs (k, H - k); Z[k] = src[(k mod R) LZ + k / R]
    float2* Xr = a.X + b * a.ld_X;
    const float2* wk = a.tab + a.unpack_off;
    for (int k = threadIdx.x; k <= H / 2; k += kMixedThreads) {
        const int km = k == 0 ? 0 : H - k;
        const float2 A = src[(k % R) * LZ + k / R];
        const float2 B = src[(km % R) * LZ + km / R];
        unpack_pair_mixed(Xr, k, H, A, B, __ldg(wk + k));
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
        // table: pre-twiddles [R][LZ] | pass twiddles | roots of 3, 5, 7 | unpack
        int pass = 0, ns = 1;
        for (int r : rad) {
            if (ns > 1) pass += (r - 1) * ns;
            ns *= r;
        }
        p->pre_off = 0;
        p->pass_off = (int)H;
        p->root_off = p->pass_off + pass;
        p->unpack_off = p->root_off + 15;
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
    int q = p.root_off;
    for (int r : {3, 5, 7})
        for (int i = 0; i < r; ++i) host[q++] = w(i, r);
    for (int64_t k = 0; k <= H / 2; ++k) host[p.unpack_off + k] = w(k, 2 * H);
}

cudaError_t mixed_launch(const MixedPlan& p, const float* x, int64_t batch, int n, int64_t ld_x, const float2* tab,
                         float2* X, int64_t ld_X, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    MixedArgs a = {};
    a.x = x; a.batch = batch; a.n = n; a.ld_x = ld_x; a.X = X; a.ld_X = ld_X;
    a.H = p.H; a.LZ = p.LZ; a.R = p.R; a.npass = (int)p.radix.size();
    for (size_t i = 0; i < p.radix.size(); ++i) a.radix[i] = p.radix[i];
    a.tab = tab;
    a.pre_off = p.pre_off; a.pass_off = p.pass_off; a.root_off = p.root_off; a.unpack_off = p.unpack_off;
    cudaError_t e = cudaFuncSetAttribute(k_fft_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    k_fft_mixed<<<(unsigned)batch, kMixedThreads, p.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace spec
