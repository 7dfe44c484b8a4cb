// k_gemm.cu -- the chirp-z transform as a dense product on the tensor cores.
//
// Eq. 11 on the unit circle is a matrix product: with
//   Z[k][n] = z_k^{-n} = e^{-j 2 pi (f1 + k step) n / fs}   (Eq. 16-23, A_0 = W_0 = 1)
// the spectra of a batch are X = x Z^T.  In real arithmetic that is
//   out[b][2k] = sum_n x[b][n] cos(2 pi phi_kn),  out[b][2k+1] = -sum_n x[b][n] sin(2 pi phi_kn),
// a [B x N] . [N x 2M] GEMM whose output rows are the complex64 spectra.
// The paper evaluates the CZT only by Bluestein's method; this form trades
// the FFTs for tensor-core work and wins when N and M are moderate.
//
// Precision.  x is scaled per row by a power of two s (so max |x s| < 2^15)
// and Z by 2^14, then each is split into two FP16 parts,
//   x s = xh + xl 2^-11,   Z 2^14 = Zh + Zl 2^-11,
// so that x s Z 2^14 = xh Zh + (xh Zl + xl Zh) 2^-11 + O(2^-22).  Three FP16
// products accumulate in FP32 in two tensor-memory accumulators,
//   D1 = sum xh Zh,  D2 = sum (xh Zl + xl Zh),  out = (D1 + D2 2^-11) 2^-14 / s,
// which keeps the result within a few 1e-7 of the FP64 value -- the accuracy
// of the FP32 Bluestein path.  The one-product form (D1 only) is about 1e-3.
//
// Kernel: persistent, one CTA per SM, 128 x 128 output tiles.
//   warp 0, one thread  TMA loads of the xh, xl, Zh, Zl tiles (128 rows x 64
//                       FP16, 128-byte swizzle) into a 3-stage ring;
//   warp 1, one thread  tcgen05.mma (kind::f16, M = N = 128, K = 16) into
//                       two double-buffered accumulator pairs in TMEM;
//   warps 2-5           epilogue: tcgen05.ld, combine, scale, store.
// Every mbarrier wait is bounded in time; a wait that gives up sets the
// context's status word, and the CTA drains its copies and products in
// flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "mbarrier.cuh"
#include "spec_internal.h"

namespace spec {
namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 3;
constexpr int TILE_A = BM * BK * 2;               // bytes of one FP16 part of an x tile
constexpr int TILE_B = BN * BK * 2;
constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;
constexpr int THREADS = 192;
// with the FP16 split fused into the product: four more warps convert each
// staged FP32 x tile in place into the parts the tensor cores read
constexpr int THREADS_FUSED = 448;
constexpr int NCONV = THREADS_FUSED - 192;       // converter threads (8 warps)
constexpr int CONV0 = 192;                        // first converter thread
constexpr uint32_t TMEM_COLS = 512;               // 2 buffers x (D1, D2) x 128 columns
// epilogue staging for bulk tensor stores: per epilogue warp two 32 x 32
// float boxes (4 KB each, rows of 128 bytes in the 128-byte swizzle)
constexpr int OUT_BOX = 32 * 32 * 4;
constexpr int OUT_BYTES = 4 * 2 * OUT_BOX;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + OUT_BYTES + 1024 + 256;

// Instruction descriptor, kind::f16: FP32 accumulate (bits 4-5 = 1), A and B
// FP16 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
// The same with A and B BF16 (format 1 at bits 7-9 and 10-12; both operands
// always share one format)
constexpr uint32_t kIdescBf16 = kIdesc | (1u << 7) | (1u << 10);

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Bulk tensor store of a shared-memory box to global memory (bulk group).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"((uint64_t)map),
                 "r"(smem_u32(src)), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most N bulk groups still reading their shared-memory source
template <int N> __device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy shared-memory writes visible to the asynchronous proxy
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 64 FP16 (128 B), 8-row groups 1024 B apart (stride byte offset),
// descriptor version 1, layout type 2 (SWIZZLE_128B).  Address >> 4 in bits
// 0-13; a K step of 16 elements advances the address by 32 B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate,
                                         uint32_t idesc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 consecutive 32-bit columns of tensor memory, one lane per thread
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct GemmArgs {
    int64_t rows;              // B
    int cols;                  // 2M
    int kblocks;               // padded N / 64
    int ntn;                   // column tiles
    int64_t tiles;
    int terms;                 // 3 (FP16 split), 1 (one FP16 product) or -1 (one BF16 product)
    const int* row_pow;        // per row: log2 of its scale s
    const int* col_pow;        // per output bin k: log2 of Z's column scale (spiral contours), or null
    float* out;
    int64_t ld_out;            // floats
    int vec4;                  // rows and base 16-byte aligned: 16-byte stores
    int tma_out;               // mOut describes out: bulk tensor stores from shared memory
    unsigned* status;
    uint64_t timeout_ns;
};

// Barrier 1 of the NCONV converter threads, returning the OR of `pred` over them.
__device__ __forceinline__ bool bar_or_conv(bool pred) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "n"(NCONV)
        : "memory");
    return r != 0;
}

// FUSED converter (NCONV = 256 threads, ct < 256): for every stage in the
// order the producer fills them, wait for the FP32 x box (128 rows x 64
// samples, rows of 256 bytes), scale row r by 2^row_pow[r] and split it into
// the FP16 parts (the arithmetic of k_gemm_split_x, so the parts are the same
// bits), then, once all converter threads have read the box, write the parts
// over it in the K-major 128-byte-swizzled layout the product reads (part h
// at the stage's A area, part l at A + TILE_A), make the writes visible to the
// tensor cores and arrive on conv.  Thread ct owns 16-byte chunk ct mod 8 of
// rows ct/8 + 32 i (i < 4): a quarter-warp reads 128 contiguous bytes and
// writes one swizzled 128-byte row, both without bank conflicts.
__device__ __forceinline__ void convert_stages(const GemmArgs& a, uint8_t* base, uint64_t* full, uint64_t* conv,
                                               const Guard& g, int ct) {
    constexpr int ROWS = NCONV / 8, PER = BM / ROWS;        // 32 rows a sweep, 4 sweeps
    const int ch = ct & 7;
    const int hsel = (ch >> 2) & 1;              // which 16-byte half is read first (spreads the banks)
    int stage = 0;
    uint32_t ph = 0;
    for (int64_t tile = blockIdx.x; tile < a.tiles; tile += gridDim.x) {
        const int64_t m0 = (tile / a.ntn) * BM;
        float sc[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int64_t row = m0 + (ct >> 3) + ROWS * i;
            sc[i] = row < a.rows ? ldexpf(1.0f, a.row_pow[row]) : 0.f;
        }
        for (int kb = 0; kb < a.kblocks; ++kb) {
            // a wait that gives up is acted on by all converter threads
            // together (at the barrier below), so that none is left waiting
            const bool okw = wait_bounded(full + stage, ph, g);
            uint8_t* sa = base + stage * STAGE_BYTES;
            uint4 hi[PER], lo[PER];
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int r = (ct >> 3) + ROWS * i;
                const float4* src = reinterpret_cast<const float4*>(sa + r * 256 + ch * 32);
                const float4 f0 = src[hsel], f1 = src[hsel ^ 1];
                const float4 q0 = hsel ? f1 : f0, q1 = hsel ? f0 : f1;
                const float2 xv[4] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(q1.x, q1.y),
                                      make_float2(q1.z, q1.w)};
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 v = make_float2(xv[e].x * sc[i], xv[e].y * sc[i]);
                    if (a.terms < 0) {
                        const __nv_bfloat162 b2 = __floats2bfloat162_rn(v.x, v.y);
                        hw[e] = *reinterpret_cast<const uint32_t*>(&b2);
                        lw[e] = 0;
                    } else {
                        const __half2 h2 = __floats2half2_rn(v.x, v.y);
                        const float2 hb = __half22float2(h2);
                        const __half2 l2 = __floats2half2_rn((v.x - hb.x) * 2048.f, (v.y - hb.y) * 2048.f);
                        hw[e] = *reinterpret_cast<const uint32_t*>(&h2);
                        lw[e] = *reinterpret_cast<const uint32_t*>(&l2);
                    }
                }
                hi[i] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                lo[i] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
            // every converter thread has read the box before any part
            // overwrites it; the same barrier ORs the threads' wait failures
            if (bar_or_conv(!okw)) return;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int r = (ct >> 3) + ROWS * i;
                const int off = (r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4);
                *reinterpret_cast<uint4*>(sa + off) = hi[i];
                if (a.terms == 3) *reinterpret_cast<uint4*>(sa + TILE_A + off) = lo[i];
            }
            fence_async_shared();
            mbar_arrive(conv + stage);
            if (++stage == STAGES) { stage = 0; ph ^= 1u; }
        }
    }
}

template <bool FUSED>
__global__ void __launch_bounds__(FUSED ? THREADS_FUSED : THREADS, 1)
    k_czt_gemm(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
               const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
               const __grid_constant__ CUtensorMap mOut, GemmArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* obuf = base + STAGES * STAGE_BYTES;               // 1024-byte aligned
    uint64_t* full = (uint64_t*)(obuf + OUT_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* done = tempty + 2;
    uint64_t* conv = done + 1;                   // FUSED: stage converted (NCONV arrivals)
    uint32_t* tmem_slot = (uint32_t*)(conv + STAGES);
    int* abort_flag = (int*)(tmem_slot + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
            mbar_init(conv + s, NCONV);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(tfull + i, 1);
            mbar_init(tempty + i, 128);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const Guard g{abort_flag, a.status, a.timeout_ns};
    // FUSED: the A part of a stage is one 128 x 64 FP32 box of x (both FP16
    // parts' space); otherwise the FP16 parts made by k_gemm_split_x
    const uint32_t stage_tx = FUSED ? (uint32_t)(2 * TILE_A + (a.terms == 3 ? 2 : 1) * TILE_B)
                                    : a.terms == 3 ? (uint32_t)STAGE_BYTES : (uint32_t)(TILE_A + TILE_B);
    const uint32_t idesc = a.terms < 0 ? kIdescBf16 : kIdesc;

    if (warp == 0) {
        if (lane == 0) {
            // producer
            int stage = 0;
            uint32_t ph = 0;
            int issued_ph[STAGES];
            for (int s = 0; s < STAGES; ++s) issued_ph[s] = -1;
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < a.tiles; tile += gridDim.x) {
                const int m0 = (int)(tile / a.ntn) * BM;
                const int n0 = (int)(tile % a.ntn) * BN;
                for (int kb = 0; kb < a.kblocks; ++kb) {
                    if (!wait_bounded(empty + stage, ph ^ 1u, g)) { ok = false; break; }
                    uint8_t* sa = base + stage * STAGE_BYTES;
                    mbar_expect_tx(full + stage, stage_tx);
                    tma_load_2d(sa, &mAh, full + stage, kb * BK, m0);
                    tma_load_2d(sa + 2 * TILE_A, &mBh, full + stage, kb * BK, n0);
                    if (a.terms == 3) {
                        if (!FUSED) tma_load_2d(sa + TILE_A, &mAl, full + stage, kb * BK, m0);
                        tma_load_2d(sa + 2 * TILE_A + TILE_B, &mBl, full + stage, kb * BK, n0);
                    }
                    issued_ph[stage] = (int)ph;
                    if (++stage == STAGES) { stage = 0; ph ^= 1u; }
                }
            }
            // no copy may still be landing in shared memory when the CTA exits
            const Guard g2{abort_flag, a.status, a.timeout_ns};
            for (int s = 0; s < STAGES; ++s) {
                if (issued_ph[s] < 0) continue;
                const uint64_t t0 = gtime();
                while (!mbar_try_wait(full + s, (uint32_t)issued_ph[s]) && gtime() - t0 < g2.timeout_ns) {
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            int stage = 0;
            uint32_t ph = 0;
            int acc = 0;
            uint32_t aph = 0;
            bool ok = true;
            bool any = false;
            for (int64_t tile = blockIdx.x; ok && tile < a.tiles; tile += gridDim.x) {
                if (!wait_bounded(tempty + acc, aph ^ 1u, g)) break;
                tc_fence_after();
                const uint32_t d1 = tmem + (uint32_t)(acc * 256);
                const uint32_t d2 = d1 + 128;
                for (int kb = 0; kb < a.kblocks; ++kb) {
                    if (!wait_bounded((FUSED ? conv : full) + stage, ph, g)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(base + stage * STAGE_BYTES);
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
                        const uint64_t ah = sw128_desc(sa + ks * 32);
                        const uint64_t bh = sw128_desc(sa + 2 * TILE_A + ks * 32);
                        const uint32_t accum = (kb | ks) != 0;
                        umma_f16(d1, ah, bh, accum, idesc);
                        if (a.terms == 3) {
                            const uint64_t al = sw128_desc(sa + TILE_A + ks * 32);
                            const uint64_t bl = sw128_desc(sa + 2 * TILE_A + TILE_B + ks * 32);
                            umma_f16(d2, ah, bl, accum, idesc);
                            umma_f16(d2, al, bh, 1u, idesc);
                        }
                    }
                    any = true;
                    umma_commit(empty + stage);          // frees the stage when these products finish
                    if (++stage == STAGES) { stage = 0; ph ^= 1u; }
                }
                if (!ok) break;
                umma_commit(tfull + acc);
                if (++acc == 2) { acc = 0; aph ^= 1u; }
            }
            // every product must be finished before the tensor memory is freed
            if (any) {
                umma_commit(done);
                const uint64_t t0 = gtime();
                while (!mbar_try_wait(done, 0) && gtime() - t0 < a.timeout_ns) {
                }
            }
        }
    } else if (FUSED && warp >= CONV0 / 32) {
        convert_stages(a, base, full, conv, g, threadIdx.x - CONV0);
    } else {
        // epilogue, warps 2..5: warp w reads TMEM lanes 32 (w % 4) .. + 31
        const int q = warp & 3;
        int acc = 0;
        uint32_t aph = 0;
        int nbox = 0;                                    // boxes this warp has stored
        for (int64_t tile = blockIdx.x; tile < a.tiles; tile += gridDim.x) {
            if (!wait_bounded(tfull + acc, aph, g)) break;
            tc_fence_after();
            const int64_t row = (tile / a.ntn) * BM + q * 32 + lane;
            const int n0 = (int)(tile % a.ntn) * BN;
            const bool live = row < a.rows;
            const int rp = live ? a.row_pow[row] : 0;
            const float scale = live ? ldexpf(1.0f, -14 - rp) : 0.f;
            float* orow = a.out + (live ? row : 0) * a.ld_out;
            const uint32_t tbase = tmem + (uint32_t)(acc * 256) + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t r1[32], r2[32];
                tmem_ld32(tbase + c * 32, r1);
                if (a.terms == 3) tmem_ld32(tbase + 128 + c * 32, r2);
                tmem_ld_wait();
                if (a.tma_out) {
                    // stage the warp's 32 x 32 box (row = lane, 128-byte
                    // swizzle: 16-byte chunk u of row r at u ^ (r mod 8)) and
                    // store it with one bulk tensor copy; rows beyond the
                    // batch and columns beyond 2M are clipped by the copy
                    uint8_t* box = obuf + (size_t)(q * 2 + (nbox & 1)) * OUT_BOX;
                    if (nbox >= 2) {
                        if (lane == 0) bulk_wait_read<1>();         // this buffer's last store has read it
                        __syncwarp();
                    }
                    const int colb = n0 + c * 32;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        float v[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            v[e] = __uint_as_float(r1[4 * u + e]);
                            if (a.terms == 3) v[e] = fmaf(__uint_as_float(r2[4 * u + e]), 4.8828125e-4f, v[e]);
                        }
                        const int k0 = (colb + 4 * u) >> 1;        // output bins of the chunk's columns
                        const float s0 = a.col_pow && live ? ldexpf(1.0f, -14 - rp + a.col_pow[min(k0, a.cols / 2 - 1)]) : scale;
                        const float s1 = a.col_pow && live ? ldexpf(1.0f, -14 - rp + a.col_pow[min(k0 + 1, a.cols / 2 - 1)]) : scale;
                        *(float4*)(box + lane * 128 + ((u ^ (lane & 7)) << 4)) =
                            make_float4(v[0] * s0, v[1] * s0, v[2] * s1, v[3] * s1);
                    }
                    fence_async_shared();
                    __syncwarp();
                    if (lane == 0) {
                        // a box wholly past the batch is not stored (only
                        // boxes that start inside the tensor are issued)
                        const int64_t row0 = (tile / a.ntn) * BM + q * 32;
                        if (row0 < a.rows && colb < a.cols) tma_store_2d(&mOut, box, colb, (int)row0);
                        bulk_commit();
                    }
                    ++nbox;
                } else if (live && a.vec4 && n0 + c * 32 + 32 <= a.cols) {
                    // whole 32-column chunk inside the output: 16-byte stores
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const int col = n0 + c * 32 + j;
                        float v[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            v[u] = __uint_as_float(r1[j + u]);
                            if (a.terms == 3) v[u] = fmaf(__uint_as_float(r2[j + u]), 4.8828125e-4f, v[u]);   // 2^-11
                        }
                        const float s0 = a.col_pow ? ldexpf(1.0f, -14 - rp + a.col_pow[col >> 1]) : scale;
                        const float s1 = a.col_pow ? ldexpf(1.0f, -14 - rp + a.col_pow[(col >> 1) + 1]) : scale;
                        *(float4*)(orow + col) = make_float4(v[0] * s0, v[1] * s0, v[2] * s1, v[3] * s1);
                    }
                } else if (live) {
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        const int col = n0 + c * 32 + j;
                        float v0 = __uint_as_float(r1[j]), v1 = __uint_as_float(r1[j + 1]);
                        if (a.terms == 3) {
                            v0 = fmaf(__uint_as_float(r2[j]), 4.8828125e-4f, v0);          // 2^-11
                            v1 = fmaf(__uint_as_float(r2[j + 1]), 4.8828125e-4f, v1);
                        }
                        if (col < a.cols) {
                            // off the unit circle Z's column k = col/2 was scaled by 2^-col_pow[k]
                            const float sc = a.col_pow ? ldexpf(1.0f, -14 - rp + a.col_pow[col >> 1]) : scale;
                            *(float2*)(orow + col) = make_float2(v0 * sc, v1 * sc);
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(tempty + acc);
            if (++acc == 2) { acc = 0; aph ^= 1u; }
        }
        // every bulk store of this warp complete before the CTA (and its
        // shared memory) goes away
        if (a.tma_out && lane == 0) bulk_wait_all();
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// One warp per row: row scale s = 2^p with max |x| s < 2^15, then the FP16
// parts xh = fp16(x s), xl = fp16((x s - xh) 2^11), zero-padded to np.
__global__ void k_gemm_split_x(const float* x, int64_t batch, int n, int64_t ld_x, int np, __half* xh, __half* xl,
                               int* row_pow, int terms) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (row >= batch) return;
    const float* xr = x + row * ld_x;
    float mx = 0.f;
    for (int i = lane; i < n; i += 32) mx = fmaxf(mx, fabsf(xr[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f && mx <= 3.4e38f) frexpf(mx, &e);      // mx < 2^e
    const int p = min(127, 15 - e);
    __half* hr = xh + row * np;
    __half* lr = xl + row * np;
    for (int i = lane; i < np; i += 32) {
        const float v = i < n ? ldexpf(xr[i], p) : 0.f;
        if (terms < 0) {
            // one BF16 part, stored in the same 16-bit slots
            const __nv_bfloat16 bh = __float2bfloat16_rn(v);
            hr[i] = __ushort_as_half(__bfloat16_as_ushort(bh));
            continue;
        }
        const __half h = __float2half_rn(v);
        hr[i] = h;
        if (terms == 3) lr[i] = __float2half_rn((v - __half2float(h)) * 2048.f);
    }
    if (lane == 0) row_pow[row] = p;
}

// The row exponents alone (for the product with the split fused in): one
// warp per row, p = min(127, 15 - e) with max |x| < 2^e, as k_gemm_split_x.
__global__ void k_gemm_row_pow(const float* x, int64_t batch, int n, int64_t ld_x, int* row_pow, int v4) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x % 32;
    if (row >= batch) return;
    const float* xr = x + row * ld_x;
    float mx = 0.f;
    if (v4) {                                    // n, the rows and x all 16-byte multiples
        const float4* x4 = reinterpret_cast<const float4*>(xr);
        for (int i = lane; i < n / 4; i += 32) {
            const float4 v = __ldg(x4 + i);
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
    } else {
        for (int i = lane; i < n; i += 32) mx = fmaxf(mx, fabsf(__ldg(xr + i)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f && mx <= 3.4e38f) frexpf(mx, &e);
    if (lane == 0) row_pow[row] = min(127, 15 - e);
}

// Z rows c < 2M (cos for c = 2k, -sin for c = 2k+1) at the exact phase
// A n + B k n (64-bit fixed point, cycles), scaled by 2^14 and split (or, for
// the BF16 form, rounded once to BF16 into zh; zl then holds zeros).
__global__ void k_gemm_build_z(int m, int n, int np, uint64_t A, uint64_t B, __half* zh, __half* zl, int bf16) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)2 * m * np) return;
    const int c = (int)(idx / np);
    const int i = (int)(idx % np);
    const uint64_t k = (uint64_t)(c >> 1);
    double v = 0.0;
    if (i < n) {
        const uint64_t ph = A * (uint64_t)i + B * (k * (uint64_t)i);
        const double cyc = (double)(int64_t)ph * 5.421010862427522e-20;   // * 2^-64
        double s, co;
        sincospi(2.0 * cyc, &s, &co);
        v = (c & 1) ? -s : co;
    }
    v *= 16384.0;
    if (bf16) {
        zh[idx] = __ushort_as_half(__bfloat16_as_ushort(__double2bfloat16(v)));
        zl[idx] = __float2half_rn(0.f);
        return;
    }
    const __half h = __float2half_rn((float)v);
    zh[idx] = h;
    zl[idx] = __float2half_rn((float)((v - (double)__half2float(h)) * 2048.0));
}

// Z off the unit circle (Eq. 16-17 with A_0, W_0 != 1): Z[k][n] = A^{-n} W^{kn},
// magnitude exp(-n ln A_0 + k n ln W_0), divided by 2^col_pow[k] (the column's
// largest magnitude rounded up to a power of two), then scaled and split as
// the unit-circle table.
__global__ void k_gemm_build_z_spiral(int m, int n, int np, uint64_t A, uint64_t B, double la, double lw,
                                      const int* col_pow, __half* zh, __half* zl) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)2 * m * np) return;
    const int c = (int)(idx / np);
    const int i = (int)(idx % np);
    const uint64_t k = (uint64_t)(c >> 1);
    double v = 0.0;
    if (i < n) {
        const uint64_t ph = A * (uint64_t)i + B * (k * (uint64_t)i);
        const double cyc = (double)(int64_t)ph * 5.421010862427522e-20;   // * 2^-64
        double s, co;
        sincospi(2.0 * cyc, &s, &co);
        const double mag = exp(-la * (double)i + lw * (double)(k * (uint64_t)i) -
                               0.6931471805599453 * (double)col_pow[k]);
        v = mag * ((c & 1) ? -s : co);
    }
    v *= 16384.0;
    const __half h = __float2half_rn((float)v);
    zh[idx] = h;
    zl[idx] = __float2half_rn((float)((v - (double)__half2float(h)) * 2048.0));
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
    });
    return fn;
}

// 2-D FP16 tensor [rows][np], boxes of 128 rows x 64 columns, 128-byte swizzle
// Output [rows][cols] float32 at a row pitch of ld floats, stored in 32 x 32
// boxes with the 128-byte swizzle (the epilogue's staging layout).
bool make_out_map(CUtensorMap* map, float* ptr, int64_t rows, int cols, int64_t ld) {
    EncodeFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// x itself, [rows][n] float32 at a row pitch of ld floats, in 128 x 64
// boxes without swizzle (the converter reads 256-byte rows); samples past n
// read as zeros.
bool make_x_map(CUtensorMap* map, const float* ptr, int64_t rows, int64_t n, int64_t ld) {
    EncodeFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {BK, BM};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_map(CUtensorMap* map, const __half* ptr, int64_t rows, int np) {
    EncodeFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)np, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)np * 2};
    const cuuint32_t box[2] = {BK, 128};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void*)ptr, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// SPEC_GEMM_TMA_OUT=0 keeps the per-thread 16-byte stores (for comparison)
bool tma_out_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("SPEC_GEMM_TMA_OUT");
        return !(e && std::atoi(e) == 0);
    }();
    return on;
}

}  // namespace

int gemm_padded_n(int64_t n) { return (int)((n + BK - 1) / BK * BK); }

size_t gemm_z_bytes(int64_t n, int64_t m) { return (size_t)2 * (2 * m) * gemm_padded_n(n) * sizeof(__half); }

size_t gemm_work_bytes(int64_t batch, int64_t n) {
    const size_t np = (size_t)gemm_padded_n(n);
    return ((size_t)2 * batch * np * sizeof(__half) + 255) / 256 * 256 + (size_t)batch * sizeof(int);
}

cudaError_t gemm_build_z(int64_t n, int64_t m, uint64_t A, uint64_t B, void* z, cudaStream_t st, bool bf16) {
    const int np = gemm_padded_n(n);
    __half* zh = (__half*)z;
    __half* zl = zh + (size_t)2 * m * np;
    const int64_t total = (int64_t)2 * m * np;
    k_gemm_build_z<<<(unsigned)((total + 255) / 256), 256, 0, st>>>((int)m, (int)n, np, A, B, zh, zl, bf16 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t gemm_build_z_spiral(int64_t n, int64_t m, uint64_t A, uint64_t B, double la, double lw,
                                const int* col_pow, void* z, cudaStream_t st) {
    const int np = gemm_padded_n(n);
    __half* zh = (__half*)z;
    __half* zl = zh + (size_t)2 * m * np;
    const int64_t total = (int64_t)2 * m * np;
    k_gemm_build_z_spiral<<<(unsigned)((total + 255) / 256), 256, 0, st>>>((int)m, (int)n, np, A, B, la, lw, col_pow,
                                                                            zh, zl);
    return cudaGetLastError();
}

cudaError_t gemm_split_launch(const float* x, int64_t batch, int64_t n, int64_t ld_x, int terms, void* work,
                              cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    const int np = gemm_padded_n(n);
    __half* xh = (__half*)work;
    __half* xl = xh + (size_t)batch * np;
    int* row_pow = (int*)((uint8_t*)work + ((size_t)2 * batch * np * sizeof(__half) + 255) / 256 * 256);
    k_gemm_split_x<<<(unsigned)((batch + 7) / 8), 256, 0, st>>>(x, batch, (int)n, ld_x, np, xh, xl, row_pow, terms);
    return cudaGetLastError();
}

bool gemm_fused_ok(const float* x, int64_t ld_x) {
    return (reinterpret_cast<uintptr_t>(x) & 15) == 0 && (ld_x & 3) == 0;
}

cudaError_t gemm_rowpow_launch(const float* x, int64_t batch, int64_t n, int64_t ld_x, void* work, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    const int np = gemm_padded_n(n);
    int* row_pow = (int*)((uint8_t*)work + ((size_t)2 * batch * np * sizeof(__half) + 255) / 256 * 256);
    const bool v4 = (n & 3) == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0 && (ld_x & 3) == 0;
    k_gemm_row_pow<<<(unsigned)((batch + 7) / 8), 256, 0, st>>>(x, batch, (int)n, ld_x, row_pow, v4 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t gemm_mul_launch(int64_t batch, int64_t n, int64_t m, int terms, const void* z, const void* work,
                            float2* X, int64_t ld_X, unsigned* status, int sms, uint64_t timeout_ns,
                            cudaStream_t st, const int* col_pow, const float* x, int64_t ld_x) {
    if (batch == 0) return cudaSuccess;
    const int np = gemm_padded_n(n);
    const __half* xh = (const __half*)work;
    const __half* xl = xh + (size_t)batch * np;
    const int* row_pow =
        (const int*)((const uint8_t*)work + ((size_t)2 * batch * np * sizeof(__half) + 255) / 256 * 256);
    const __half* zh = (const __half*)z;
    const __half* zl = zh + (size_t)2 * m * np;
    const bool fused = x != nullptr;
    CUtensorMap mAh, mAl, mBh, mBl;
    if (fused) {
        if (!make_x_map(&mAh, x, batch, n, ld_x)) return cudaErrorInvalidValue;
        mAl = mAh;
    } else if (!make_map(&mAh, xh, batch, np) || !make_map(&mAl, xl, batch, np)) {
        return cudaErrorInvalidValue;
    }
    if (!make_map(&mBh, zh, 2 * m, np) || !make_map(&mBl, zl, 2 * m, np)) return cudaErrorInvalidValue;
    GemmArgs a = {};
    a.rows = batch;
    a.cols = (int)(2 * m);
    a.kblocks = np / BK;
    a.ntn = (int)((2 * m + BN - 1) / BN);
    a.tiles = (batch + BM - 1) / BM * a.ntn;
    a.terms = terms;
    a.row_pow = row_pow;
    a.col_pow = col_pow;
    a.out = (float*)X;
    a.ld_out = 2 * ld_X;
    a.vec4 = ((reinterpret_cast<uintptr_t>(X) & 15) == 0 && (a.ld_out & 3) == 0) ? 1 : 0;
    CUtensorMap mOut;
    std::memset(&mOut, 0, sizeof(mOut));
    a.tma_out = (a.vec4 && tma_out_enabled() && make_out_map(&mOut, a.out, batch, a.cols, a.ld_out)) ? 1 : 0;
    a.status = status;
    a.timeout_ns = timeout_ns;
    const void* kf = fused ? (const void*)k_czt_gemm<true> : (const void*)k_czt_gemm<false>;
    cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(a.tiles, (int64_t)std::max(1, sms));
    if (fused) k_czt_gemm<true><<<(unsigned)grid, THREADS_FUSED, SMEM_BYTES, st>>>(mAh, mAl, mBh, mBl, mOut, a);
    else k_czt_gemm<false><<<(unsigned)grid, THREADS, SMEM_BYTES, st>>>(mAh, mAl, mBh, mBl, mOut, a);
    return cudaGetLastError();
}

// A wait that nothing will end: one mbarrier that expects an arrival no one
// makes, waited on with the same bounded loop as the GEMM.  Exercises the
// timeout path (status word set, clean return).
__global__ void k_wait_selftest(unsigned* status, uint64_t timeout_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        mbar_init_fence();
    }
    __syncthreads();
    const Guard g{&abort_flag, status, timeout_ns};
    if (threadIdx.x == 0) wait_bounded(&bar, 0, g);
    __syncthreads();
}

cudaError_t wait_selftest_launch(unsigned* status, uint64_t timeout_ns, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(status, timeout_ns);
    return cudaGetLastError();
}

}  // namespace spec
