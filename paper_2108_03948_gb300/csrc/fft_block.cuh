// fft_block.cuh -- device building blocks shared by the transform kernels.
//
// * complex helpers; a complex float2 is also a packed FP32 pair, so complex
//   additions are single add/sub.rn.f32x2 instructions;
// * in-register DFTs of size 2, 4, 8, 16;
// * BlockFFT: a power-of-two complex FFT executed by a group of T threads,
//   each holding E = LF/T elements in registers.  Before and after the
//   transform thread t holds elements t + T*i (i < E) in natural order, so
//   loads, pointwise products and stores need no shared-memory staging; only
//   the Stockham passes in between exchange through shared memory.  The
//   inter-pass twiddles come from a table generated once in float64, laid
//   out so that the lanes of a warp read consecutive entries;
// * exact phases: a phase in cycles is kept as a 64-bit fixed-point fraction,
//   so products such as (b/2) n^2 are reduced modulo one cycle exactly by
//   integer wrap-around before any floating-point trig call.
//
// The FFT itself is the DFT of Section 2.1, Eq. 2 (forward sign e^{-j...});
// the inverse (used by Bluestein's convolution, Eq. 15) flips the sign.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spec {

// ------------------------------------------------------------ packed pairs --
__device__ __forceinline__ uint64_t pk(float2 a) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 upk(uint64_t r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(d);
}

// ---------------------------------------------------------------- complex --
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return add2(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return sub2(a, b); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return mul2(a, make_float2(s, s)); }

// multiply by e^{-j pi/2} (forward) or e^{+j pi/2} (inverse)
template <bool INV> __device__ __forceinline__ float2 rot90(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// e^{sign j 2 pi ph/2^64}: `ph` is a phase in cycles as a 64-bit fixed-point
// fraction.  Its top 24 bits q (a signed cycle fraction q 2^-24, exact in
// float) go through sincospif; the remainder r = ph - q 2^40, below 2^40
// (an angle under 2 pi 2^-24), is applied to first order (the neglected
// second-order term is below 1e-13), so the result is accurate to the float
// rounding of cos and sin (below 1e-7 absolute) whatever the size of the
// original phase.  Only 32-bit integer to
// float conversions are used: the 64-bit ones run on the (slow) FP64 pipe.
__device__ __forceinline__ float2 unit_fixed(uint64_t ph, bool negative) {
    const int32_t q = (int32_t)((int64_t)ph >> 40);            // [-2^23, 2^23)
    const uint64_t r = ph - ((uint64_t)(int64_t)q << 40);       // [0, 2^40)
    const float xf = (float)q * 1.1920928955078125e-07f;       // * 2^-23 (half-cycles)
    const float xr = (float)(int32_t)(r >> 9) * 1.7439342e-16f;  // * 2^9 2^-64 2 pi (radians)
    float sn, cs;
    sincospif(xf, &sn, &cs);
    const float re = fmaf(-xr, sn, cs);
    const float im = fmaf(xr, cs, sn);
    return negative ? make_float2(re, -im) : make_float2(re, im);
}

// Same phase through the hardware sine and cosine (__sincosf, absolute error
// about 4e-7 for arguments in [-pi, pi], which the fixed-point reduction
// guarantees), with the same first-order remainder: for chirps evaluated in a
// kernel, where the library call's cost matters.
__device__ __forceinline__ float2 unit_fast(uint64_t ph, bool negative) {
    const int32_t q = (int32_t)((int64_t)ph >> 40);
    const uint64_t r = ph - ((uint64_t)(int64_t)q << 40);
    const float ang = (float)q * 3.7450703e-07f;               // * 2 pi 2^-24 (radians)
    const float xr = (float)(int32_t)(r >> 9) * 1.7439342e-16f;
    float sn, cs;
    __sincosf(ang, &sn, &cs);
    const float re = fmaf(-xr, sn, cs);
    const float im = fmaf(xr, cs, sn);
    return negative ? make_float2(re, -im) : make_float2(re, im);
}

// e^{sign j 2 pi ph/2^64} evaluated in float64 (table generation only).
__device__ __forceinline__ float2 unit_fixed_f64(uint64_t ph, bool negative) {
    const double cyc = (double)(int64_t)ph * 5.421010862427522e-20;   // * 2^-64
    double s, c;
    sincospi(2.0 * cyc, &s, &c);
    return make_float2((float)c, negative ? (float)-s : (float)s);
}

// ------------------------------------------------- two-lane complex pairs --
// C2 holds two independent complex numbers a and b as packed FP32 pairs:
// re = (a.x, b.x), im = (a.y, b.y).  Every operation below is one packed
// instruction per component, so a C2 costs the instructions of one complex.
struct C2 {
    float2 re, im;
};
__device__ __forceinline__ C2 c2(float2 a, float2 b) { return C2{make_float2(a.x, b.x), make_float2(a.y, b.y)}; }
__device__ __forceinline__ float2 lane_a(C2 v) { return make_float2(v.re.x, v.im.x); }
__device__ __forceinline__ float2 lane_b(C2 v) { return make_float2(v.re.y, v.im.y); }

__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return add2(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return sub2(a, b); }
__device__ __forceinline__ C2 vadd(C2 a, C2 b) { return C2{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ C2 vsub(C2 a, C2 b) { return C2{sub2(a.re, b.re), sub2(a.im, b.im)}; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ C2 vneg(C2 a) {
    return C2{mul2(a.re, make_float2(-1.f, -1.f)), mul2(a.im, make_float2(-1.f, -1.f))};
}

// o1 = t1 - j d, o3 = t1 + j d (forward); the inverse swaps them
template <bool INV> __device__ __forceinline__ void jpair(float2 t1, float2 d, float2& o1, float2& o3) {
    const float2 ds = make_float2(d.y, d.x);
    const float2 p = INV ? make_float2(-1.f, 1.f) : make_float2(1.f, -1.f);
    o1 = fma2(ds, p, t1);
    o3 = fma2(ds, make_float2(-p.x, -p.y), t1);
}
template <bool INV> __device__ __forceinline__ void jpair(C2 t1, C2 d, C2& o1, C2& o3) {
    const C2 m = C2{add2(t1.re, d.im), sub2(t1.im, d.re)};   // t1 - j d
    const C2 p = C2{sub2(t1.re, d.im), add2(t1.im, d.re)};   // t1 + j d
    o1 = INV ? p : m;
    o3 = INV ? m : p;
}

// lane-wise complex products: C2 x C2, and one complex z times both lanes
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
    return C2{sub2(mul2(a.re, b.re), mul2(a.im, b.im)), fma2(a.re, b.im, mul2(a.im, b.re))};
}
__device__ __forceinline__ C2 cmul(float2 z, C2 b) {
    const float2 zr = make_float2(z.x, z.x), zi = make_float2(z.y, z.y);
    return C2{sub2(mul2(zr, b.re), mul2(zi, b.im)), fma2(zr, b.im, mul2(zi, b.re))};
}

// multiply by e^{-j pi/2} (forward) or e^{+j pi/2} (inverse)
template <bool INV> __device__ __forceinline__ C2 rot90(C2 a) {
    return INV ? C2{vneg(a).im, a.re} : C2{a.im, vneg(a).re};
}

// multiply by the constant c + j w
__device__ __forceinline__ float2 mulk(float2 a, float c, float w) {
    return make_float2(fmaf(a.x, c, -a.y * w), fmaf(a.x, w, a.y * c));
}
__device__ __forceinline__ C2 mulk(C2 a, float c, float w) {
    return C2{fma2(a.re, make_float2(c, c), mul2(a.im, make_float2(-w, -w))),
              fma2(a.re, make_float2(w, w), mul2(a.im, make_float2(c, c)))};
}

// Table twiddles: float2 w = c + j s (the forward twiddle) for both lane
// types; the inverse uses conj(w).  For C2 the packed pairs (c, c) and
// (s, s) are built in registers, keeping the tables small enough for L1.
template <class V> struct TwEntry;
template <> struct TwEntry<float2> { using type = float2; };
template <> struct TwEntry<C2> { using type = float2; };

template <bool INV> __device__ __forceinline__ float2 mul_tw(float2 a, float2 w) {
    return INV ? cmulc(a, w) : cmul(a, w);
}
template <bool INV> __device__ __forceinline__ C2 mul_tw_pairs(C2 a, float2 cc, float2 ss) {
    const float2 rc = mul2(a.re, cc), ic = mul2(a.im, cc);
    if (INV) return C2{fma2(a.im, ss, rc), sub2(ic, mul2(a.re, ss))};
    return C2{sub2(rc, mul2(a.im, ss)), fma2(a.re, ss, ic)};
}
template <bool INV> __device__ __forceinline__ C2 mul_tw(C2 a, float2 w) {
    return mul_tw_pairs<INV>(a, make_float2(w.x, w.x), make_float2(w.y, w.y));
}
// Twiddle stored as the packed pairs (c, c, s, s): no register shuffles.
template <bool INV> __device__ __forceinline__ C2 mul_tw(C2 a, float4 w) {
    return mul_tw_pairs<INV>(a, make_float2(w.x, w.y), make_float2(w.z, w.w));
}

// shared-memory element of a lane type
__device__ __forceinline__ void sts(float2* s, int i, float2 v) { s[i] = v; }
__device__ __forceinline__ float2 lds(const float2* s, int i, float2*) { return s[i]; }
__device__ __forceinline__ void sts(float4* s, int i, C2 v) { s[i] = make_float4(v.re.x, v.re.y, v.im.x, v.im.y); }
__device__ __forceinline__ C2 lds(const float4* s, int i, C2*) {
    const float4 q = s[i];
    return C2{make_float2(q.x, q.y), make_float2(q.z, q.w)};
}
template <class V> struct SmemT;
template <> struct SmemT<float2> { using type = float2; };
template <> struct SmemT<C2> { using type = float4; };

// ------------------------------------------------------ in-register DFTs --
template <bool INV, class V> __device__ __forceinline__ void dft2(V& a0, V& a1) {
    V t = vsub(a0, a1);
    a0 = vadd(a0, a1);
    a1 = t;
}

template <bool INV, class V> __device__ __forceinline__ void dft4(V& a0, V& a1, V& a2, V& a3) {
    const V t0 = vadd(a0, a2), t1 = vsub(a0, a2);
    const V t2 = vadd(a1, a3), d = vsub(a1, a3);
    a0 = vadd(t0, t2);
    a2 = vsub(t0, t2);
    jpair<INV>(t1, d, a1, a3);
}

constexpr float kS2 = 0.70710678118654752f;   // cos(pi/4)
constexpr float kC8 = 0.92387953251128674f;   // cos(pi/8)
constexpr float kS8 = 0.38268343236508978f;   // sin(pi/8)

// multiply by w16^P = e^{-j 2 pi P/16} (forward) or its conjugate (inverse)
template <int P, bool INV, class V> __device__ __forceinline__ V tw16(V a) {
    constexpr int Q = P & 15;
    if constexpr (Q == 0) return a;
    else if constexpr (Q == 4) return rot90<INV>(a);
    else if constexpr (Q == 8) return vneg(a);
    else if constexpr (Q == 12) return rot90<!INV>(a);
    else {
        // cos / sin of 2 pi Q/16 for Q in {1,2,3,5,6,7,9,10,11,13,14,15}
        constexpr float c = (Q == 1 || Q == 15) ? kC8 : (Q == 2 || Q == 14) ? kS2 : (Q == 3 || Q == 13) ? kS8
                          : (Q == 5 || Q == 11) ? -kS8 : (Q == 6 || Q == 10) ? -kS2 : -kC8;
        constexpr float s = (Q == 1 || Q == 7) ? kS8 : (Q == 2 || Q == 6) ? kS2 : (Q == 3 || Q == 5) ? kC8
                          : (Q == 9 || Q == 15) ? -kS8 : (Q == 10 || Q == 14) ? -kS2 : -kC8;
        // forward: e^{-j theta} = (c, -s); inverse: (c, s)
        return mulk(a, c, INV ? s : -s);
    }
}

template <bool INV, class V> __device__ __forceinline__ void dft8(V* a) {
    dft4<INV>(a[0], a[2], a[4], a[6]);
    dft4<INV>(a[1], a[3], a[5], a[7]);
    V e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    V o0 = a[1], o1 = tw16<2, INV>(a[3]), o2 = tw16<4, INV>(a[5]), o3 = tw16<6, INV>(a[7]);
    a[0] = vadd(e0, o0); a[4] = vsub(e0, o0);
    a[1] = vadd(e1, o1); a[5] = vsub(e1, o1);
    a[2] = vadd(e2, o2); a[6] = vsub(e2, o2);
    a[3] = vadd(e3, o3); a[7] = vsub(e3, o3);
}

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.
template <bool INV, class V> __device__ __forceinline__ void dft16(V* a) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
    // slot 4 k1 + n2 now holds B[n2][k1]; twiddle by w16^{n2 k1}
    a[5] = tw16<1, INV>(a[5]);  a[6] = tw16<2, INV>(a[6]);   a[7] = tw16<3, INV>(a[7]);
    a[9] = tw16<2, INV>(a[9]);  a[10] = tw16<4, INV>(a[10]); a[11] = tw16<6, INV>(a[11]);
    a[13] = tw16<3, INV>(a[13]); a[14] = tw16<6, INV>(a[14]); a[15] = tw16<9, INV>(a[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
    // slot 4 k1 + k2 holds X[k1 + 4 k2]: transpose the 4x4 (register renaming)
    V t;
    t = a[1]; a[1] = a[4]; a[4] = t;
    t = a[2]; a[2] = a[8]; a[8] = t;
    t = a[3]; a[3] = a[12]; a[12] = t;
    t = a[6]; a[6] = a[9]; a[9] = t;
    t = a[7]; a[7] = a[13]; a[13] = t;
    t = a[11]; a[11] = a[14]; a[14] = t;
}

// The same DFT when only a[0 .. 3] can be nonzero (a[4 .. 15] are ignored):
// each first-stage 4-point DFT sees one input, so it is a copy.
template <bool INV, class V> __device__ __forceinline__ void dft16_lo4(V* a) {
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) a[4 * k1 + n2] = a[n2];
    a[5] = tw16<1, INV>(a[5]);  a[6] = tw16<2, INV>(a[6]);   a[7] = tw16<3, INV>(a[7]);
    a[9] = tw16<2, INV>(a[9]);  a[10] = tw16<4, INV>(a[10]); a[11] = tw16<6, INV>(a[11]);
    a[13] = tw16<3, INV>(a[13]); a[14] = tw16<6, INV>(a[14]); a[15] = tw16<9, INV>(a[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
    V t;
    t = a[1]; a[1] = a[4]; a[4] = t;
    t = a[2]; a[2] = a[8]; a[8] = t;
    t = a[3]; a[3] = a[12]; a[12] = t;
    t = a[6]; a[6] = a[9]; a[9] = t;
    t = a[7]; a[7] = a[13]; a[13] = t;
    t = a[11]; a[11] = a[14]; a[14] = t;
}

// cos(pi k/16), k = 0 .. 8
__host__ __device__ constexpr float cos_pi16(int k) {
    return k == 0 ? 1.0f : k == 1 ? 0.98078528040323044913f : k == 2 ? 0.92387953251128675613f
         : k == 3 ? 0.83146961230254523708f : k == 4 ? 0.70710678118654752440f : k == 5 ? 0.55557023301960222474f
         : k == 6 ? 0.38268343236508977173f : k == 7 ? 0.19509032201612826785f : 0.0f;
}

// cos(pi k/32), k = 0 .. 16
__host__ __device__ constexpr float cos_pi32(int k) {
    return k == 0 ? 1.0f : k == 1 ? 0.99518472667219688624f : k == 2 ? 0.98078528040323044913f
         : k == 3 ? 0.95694033573220886494f : k == 4 ? 0.92387953251128675613f : k == 5 ? 0.88192126434835502971f
         : k == 6 ? 0.83146961230254523708f : k == 7 ? 0.77301045336273696081f : k == 8 ? 0.70710678118654752440f
         : k == 9 ? 0.63439328416364549822f : k == 10 ? 0.55557023301960222474f : k == 11 ? 0.47139673682599764856f
         : k == 12 ? 0.38268343236508977173f : k == 13 ? 0.29028467725446236764f : k == 14 ? 0.19509032201612826785f
         : k == 15 ? 0.09801714032956060199f : 0.0f;
}
// cos(pi a/32) for any integer a (period 64, even, cos(pi - x) = -cos x)
__host__ __device__ constexpr float cos_pi32_any(int a) {
    return (a % 64 + 64) % 64 <= 16 ? cos_pi32((a % 64 + 64) % 64)
         : (a % 64 + 64) % 64 <= 32 ? -cos_pi32(32 - (a % 64 + 64) % 64)
         : (a % 64 + 64) % 64 <= 48 ? -cos_pi32((a % 64 + 64) % 64 - 32)
         : cos_pi32(64 - (a % 64 + 64) % 64);
}
// e^{-j pi a/32} (sin x = cos(x - pi/2))
__host__ __device__ constexpr float2 wpi32(int a) { return float2{cos_pi32_any(a), -cos_pi32_any(a - 16)}; }
// w e^{-j pi a/32}, exact for multiples of pi/2
template <int A> __device__ __forceinline__ float2 rot_pi32(float2 w) {
    constexpr int q = ((A % 64) + 64) % 64;
    if constexpr (q == 0) return w;
    else if constexpr (q == 16) return make_float2(w.y, -w.x);
    else if constexpr (q == 32) return make_float2(-w.x, -w.y);
    else if constexpr (q == 48) return make_float2(-w.y, w.x);
    else {
        constexpr float c = cos_pi32_any(q), sn = cos_pi32_any(q - 16);
        return make_float2(fmaf(w.x, c, w.y * sn), fmaf(w.y, c, -w.x * sn));
    }
}

// 32 = 2 x 16: X[k] = E[k] + w32^k O[k], X[k + 16] = E[k] - w32^k O[k]
template <bool INV, class V> __device__ __forceinline__ void dft32(V* a) {
    V e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        e[i] = a[2 * i];
        o[i] = a[2 * i + 1];
    }
    dft16<INV>(e);
    dft16<INV>(o);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        V t = o[k];
        if (k == 8) t = rot90<INV>(t);
        else if (k != 0) {
            // w32^k = cos(pi k/16) -+ j sin(pi k/16), sin(pi k/16) = cos(pi (8-k)/16)
            const float c = k < 8 ? cos_pi16(k) : -cos_pi16(16 - k);
            const float s = k < 8 ? cos_pi16(8 - k) : cos_pi16(k - 8);
            t = mulk(t, c, INV ? s : -s);
        }
        a[k] = vadd(e[k], t);
        a[k + 16] = vsub(e[k], t);
    }
}

template <int R, bool INV, class V> __device__ __forceinline__ void dft(V* a) {
    if constexpr (R == 2) dft2<INV>(a[0], a[1]);
    else if constexpr (R == 4) dft4<INV>(a[0], a[1], a[2], a[3]);
    else if constexpr (R == 8) dft8<INV>(a);
    else if constexpr (R == 16) dft16<INV>(a);
    else if constexpr (R == 32) dft32<INV>(a);
}

// Padded shared-memory index: one spare slot per 16 keeps the stride-R writes
// of the first Stockham pass free of bank conflicts.
__host__ __device__ constexpr int pidx(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4); }
// Same with one spare slot per P (P = the radix of the first pass, whose
// stride-P writes it spreads over the banks); padded_len(n) covers it.
// (an unsigned division by the power of two P: one shift, and offsets that
// are multiples of P fold into the instruction's immediate)
template <int P> __host__ __device__ constexpr int pidx_p(int i) { return i + (int)((unsigned)i / (unsigned)P); }

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }
__host__ __device__ constexpr bool is_pow2_dev(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Barrier of the threads that share one transform's shared memory: the
// whole CTA (bar = 0), the calling warp alone (bar = -1), or the nthr threads
// (a multiple of 32) of named barrier `bar` (1 .. 7), so that transforms
// sharing a CTA do not wait for one another.  (Immediate barrier ids, so that
// the kernel reserves only the ids it uses.)
__device__ __forceinline__ void group_sync(int bar, int nthr) {
    switch (bar) {
        case -1: __syncwarp(); break;
        case 1: asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory"); break;
        case 2: asm volatile("bar.sync 2, %0;" ::"r"(nthr) : "memory"); break;
        case 3: asm volatile("bar.sync 3, %0;" ::"r"(nthr) : "memory"); break;
        case 4: asm volatile("bar.sync 4, %0;" ::"r"(nthr) : "memory"); break;
        case 5: asm volatile("bar.sync 5, %0;" ::"r"(nthr) : "memory"); break;
        case 6: asm volatile("bar.sync 6, %0;" ::"r"(nthr) : "memory"); break;
        case 7: asm volatile("bar.sync 7, %0;" ::"r"(nthr) : "memory"); break;
        default: __syncthreads();
    }
}

// ---------------------------------------------------------------- BlockFFT --
// Radix plan of an LF-point FFT with EMAX (16 or 32) elements per thread:
// radix-EMAX passes, then one pass of the remaining factor.  Pass p has
// NS = ns(p) (product of the earlier radices) and span NS R.
template <int LF, int EMAX = 16> struct FFTShape {
    static constexpr int E = LF < EMAX ? LF : EMAX;
    static constexpr int T = LF / E;
    static constexpr int LOG = ilog2c(LF);
    static constexpr int LE = ilog2c(EMAX);
    static constexpr int NPB = LOG / LE;               // full-radix passes
    static constexpr int REM = 1 << (LOG % LE);        // trailing radix
    static constexpr int NPASS = NPB + (REM > 1 ? 1 : 0);
    static constexpr int radix(int p) { return p < NPB ? EMAX : REM; }
    static constexpr int ns(int p) { return p == 0 ? 1 : ns(p - 1) * radix(p - 1); }
    // Twiddle table: pass p >= 1 holds w_{NS R}^{r k} at [off(p) + (r-1) NS + k],
    // r = 1 .. R-1, k < NS; (R-1) NS = ns(p+1) - ns(p), so off(p) = ns(p) - ns(1).
    static constexpr int tw_off(int p) { return ns(p) - ns(1); }
};

// Entries of the twiddle table of an LF-point BlockFFT: LF - EMAX for
// LF > EMAX (the first pass needs none), 0 otherwise.
__host__ __device__ constexpr int fft_twiddle_entries(int LF, int emax = 16) { return LF > emax ? LF - emax : 0; }

// LF-point FFT by T = LF/E threads, on lane type V (float2: one FFT per
// thread group; C2: two FFTs with the same twiddles, one per packed lane).
// `s` points at padded_len(LF) shared elements (SmemT<V>) owned by this FFT;
// `t` is the thread's index in [0, T); `tw` is the float64-generated twiddle
// table of this LF (TwEntry<V> by default; TWT = float4 reads the packed
// pairs (c, c, s, s) for C2 lanes; forward angles, the inverse conjugates on
// the fly).  Every thread of the CTA must call run() (it contains
// __syncthreads), including threads with dummy data.
#ifndef SPEC_TW_CHUNK
#define SPEC_TW_CHUNK 8
#endif
constexpr int kTwChunk = SPEC_TW_CHUNK;   // twiddles loaded per compiler fence

template <int LF, bool INV, class V = float2, int EMAX = 16, class TWT = typename TwEntry<V>::type> struct BlockFFT {
    using S = FFTShape<LF, EMAX>;
    using TW = TWT;
    using SM = typename SmemT<V>::type;
    static constexpr int E = S::E;
    static constexpr int T = S::T;

    template <int P>
    static __device__ __forceinline__ void compute(V (&v)[E], int t, const TW* __restrict__ tw) {
        constexpr int R = S::radix(P);
        constexpr int NS = S::ns(P);
        constexpr int NB = E / R;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            V a[R];
#pragma unroll
            for (int r = 0; r < R; ++r) a[r] = v[b + r * NB];
            if constexpr (NS > 1) {
                const int k = (t + T * b) & (NS - 1);
                const TW* twp = tw + S::tw_off(P) + k;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    // a compiler-only fence every kTwChunk twiddles keeps the
                    // loads from all being hoisted (register pressure)
                    if (r % kTwChunk == 0) asm volatile("" ::: "memory");
                    a[r] = mul_tw<INV>(a[r], __ldg(twp + (r - 1) * NS));
                }
            }
            dft<R, INV>(a);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b + r * NB] = a[r];
        }
    }

    // Write the outputs of pass P to their Stockham positions, then read the
    // thread's next inputs t + T i.
    template <int P>
    static __device__ __forceinline__ void exchange(V (&v)[E], SM* s, int t, int bar = 0, int nthr = 0) {
        constexpr int R = S::radix(P);
        constexpr int NS = S::ns(P);
        constexpr int NB = E / R;
        group_sync(bar, nthr);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = t + T * b;
            const int k = j & (NS - 1);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sts(s, pidx_p<EMAX>(base + r * NS), v[b + r * NB]);
        }
        group_sync(bar, nthr);
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = lds(s, pidx_p<EMAX>(t + T * i), (V*)nullptr);
    }

    template <int P>
    static __device__ __forceinline__ void passes(V (&v)[E], SM* s, int t, const TW* tw) {
        if constexpr (P < S::NPASS) {
            if constexpr (P > 0) exchange<P - 1>(v, s, t);
            compute<P>(v, t, tw);
            passes<P + 1>(v, s, t, tw);
        }
    }

    static __device__ __forceinline__ void run(V (&v)[E], SM* s, int t, const TW* tw) {
        passes<0>(v, s, t, tw);
    }

    // The whole FFT when only v[0 .. 3] of every thread can be nonzero (the
    // input is zero from position 4 T on): the first radix-16 pass needs no
    // twiddles and its first stage reduces to copies.
    static __device__ __forceinline__ void run_lo4(V (&v)[E], SM* s, int t, const TW* tw) {
        static_assert(E == 16 && S::radix(0) == 16, "radix-16 first pass");
        dft16_lo4<INV>(v);
        passes<1>(v, s, t, tw);
    }

    // Passes 0 .. NP-1 only (compute and the exchanges between them): the
    // caller fuses the remaining passes into its own data movement.  Thread t
    // then holds the outputs of pass NP-1 that exchange<NP-1> would store.
    // (bar, nthr): the threads that share `s` synchronise on named barrier
    // `bar` of nthr threads (bar = 0: the whole CTA)
    template <int P, int NP>
    static __device__ __forceinline__ void passes_until(V (&v)[E], SM* s, int t, const TW* tw, int bar, int nthr) {
        if constexpr (P < NP) {
            if constexpr (P > 0) exchange<P - 1>(v, s, t, bar, nthr);
            compute<P>(v, t, tw);
            passes_until<P + 1, NP>(v, s, t, tw, bar, nthr);
        }
    }
    template <int NP>
    static __device__ __forceinline__ void run_first(V (&v)[E], SM* s, int t, const TW* tw, int bar = 0,
                                                     int nthr = 0) {
        static_assert(NP >= 0 && NP <= S::NPASS, "pass count");
        passes_until<0, NP>(v, s, t, tw, bar, nthr);
    }
};

// Offset of the table of size LF in a buffer holding the tables of every
// size 2 EMAX .. LMAX (EMAX elements per thread) in increasing order.
__host__ __device__ constexpr int fft_twiddle_offset(int LF, int emax = 16) {
    return LF <= 2 * emax ? 0 : fft_twiddle_offset(LF >> 1, emax) + fft_twiddle_entries(LF >> 1, emax);
}

}  // namespace spec
