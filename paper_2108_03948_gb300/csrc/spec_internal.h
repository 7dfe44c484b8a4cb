// spec_internal.h -- launchers shared between the C-ABI layer and the
// kernel translation units.  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace spec {

// Largest per-CTA tile of complex elements for the one-pass kernels.
constexpr int kTile = 8192;

inline int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}
inline bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
inline int ilog2(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

// Placement and parameters of one trace of a ragged batch (device array,
// indexed by the trace's position in its class).  Fields a kind does not use
// are zero.
struct RaggedItem {
    int64_t x_off;     // first sample in the x pool (floats)
    int64_t out_off;   // first bin in the X pool (complex elements)
    int64_t tab_off;   // CZT: its tables (pre | V | post); Zoom: first tap in the taps pool
    int64_t u_off;     // Zoom, large path: its decimated samples in the workspace
    uint64_t A, B;     // CZT: frac(f1/fs), frac(step/(2 fs)); Zoom: A = frac(f_N/fs)
    int32_t n, m;      // samples; CZT points
    int32_t d, n_taps, lout, rs;   // Zoom
};

// Phase in cycles -> 64-bit fixed-point fraction (exact wrap-around modulo
// one cycle under unsigned multiplication).
uint64_t cycles_to_fixed(double cycles);

// ---- padded real FFT (k_fft.cu) -------------------------------------------
struct FftPlan {
    int H = 0;      // n_fft / 2 complex points after packing pairs of samples
    int LZ = 0;     // length of each residue FFT (>= ceil(n/2))
    int R = 0;      // residues H / LZ
    int C = 0;      // CTAs (cluster size) per trace
    int Rc = 0;     // residues per CTA
    int E = 0, T = 0;   // elements per thread, threads per residue FFT
    int F = 0;      // traces per CTA (C == 1 only)
    bool dual = false;  // two residues per thread (packed lanes)
    bool paired = false;  // C > 1 CTAs own residue pairs {r, R - r}: no cluster, local unpack
    bool fixed = false;   // two-lane kernel compiled for this (LZ, R) with packed tables (C == 1)
    bool clustered = false;  // one cluster of C CTAs per trace, conjugate-paired residues (k_fft_real_cluster)
    bool fused = false;      // fixed two-lane kernel with the last pass fused into the unpack (k_fft_real_fused)
    int fold = 1;            // fused: sample pairs m and m + LZ summed into one residue input (1 or 2)
    int emax = 16;      // elements per thread (16 or 32: radix of the passes)
    int trace_smem = 0; // float2 of shared memory per trace per CTA
    int threads = 0;
    size_t smem = 0;
};
// Returns false (with a reason) if the size needs a path the library lacks.
// allow_cluster = true plans k_fft_real_cluster where it has an instance;
// it measured slower than the CTA-pair kernels on GB300 (2048 traces of 8192
// samples to 65536 points: 728 against 500 us; 4096 x 4096 to 32768: 566
// against 318 us), so only the ragged autotuner times it as a candidate.
bool fft_plan(int64_t batch, int64_t n, int64_t n_fft, FftPlan* p, std::string* why, bool allow_cluster = false);
// Per-plan twiddles (pre-twiddle factors and the unpack twiddle; with
// `fixed` also the packed two-lane pre-twiddles and BlockFFT twiddles),
// float64 on the host, rounded to float.
int fft_table_entries(const FftPlan& p);
// true if k_fft_real_fused has an instance for (LZ, R) and the fold (1 or 2)
bool fft_fused_available(int LZ, int R, int fold = 1);
// The persistent fused kernel that prefetches rows with bulk copies: whole
// rows (n = 2 LZ) at 16-byte aligned addresses and pitch only.
bool fft_fused_tma_ok(const FftPlan& p, const float* x, int n, int64_t ld_x);
cudaError_t fft_fused_tma_launch(const FftPlan& p, const float* x, int64_t batch, int64_t ld_x, const float2* tab,
                                 float2* X, int64_t ld_X, unsigned* status, uint64_t timeout_ns, int sms,
                                 cudaStream_t st);
void fft_fill_table(const FftPlan& p, float2* host);
// lanes: 1 forces one FFT per thread group, otherwise the two-lane kernel is
// used where the plan allows it.
cudaError_t fft_launch(const FftPlan& p, const float* x, int64_t batch, int n, int64_t ld_x,
                       const float2* tw, const float2* tab, float2* X, int64_t ld_X, cudaStream_t st,
                       int lanes, const RaggedItem* items = nullptr);

// Pruned complex FFT with rotated store (k_fft.cu), planned in an FftPlan
// with H = K: Y[(j + shift) mod K] = FFT_K(u zero-padded)[j].
bool c2c_plan(int64_t batch, int64_t nin, int64_t K, FftPlan* p, std::string* why);
int c2c_table_entries(const FftPlan& p);
void c2c_fill_table(const FftPlan& p, float2* host);
cudaError_t c2c_launch(const FftPlan& p, const float2* u, int64_t ld_u, int nin, int64_t batch, int shift,
                       const float2* tw, const float2* tab, float2* X, int64_t ld_X, cudaStream_t st,
                       const RaggedItem* items = nullptr);

// BlockFFT twiddle tables of every size up to kMaxBlockFFT in one buffer:
// first the radix-16 layouts (sizes 32 ..), then the radix-32 ones (64 ..).
constexpr int kMaxBlockFFT = 16384;
int block_twiddle_total();
int block_twiddle_offset(int LF, int emax = 16);
void block_twiddle_fill(float2* host);
int fft_emax_for(int LF);

// ---- mixed-radix padded FFT (k_mixed.cu) -----------------------------------
// N_FFT even with N_FFT/2 = R LZ, LZ >= ceil(N/2) built from the factors 2, 3,
// 5 and 7; one CTA per trace with two shared-memory buffers of H values.
constexpr int kMixedMaxPasses = 16;
constexpr int64_t kMixedMaxH = 13312;     // 2 H complex values within one CTA's shared memory
struct MixedPlan {
    int H = 0, LZ = 0, R = 0;
    std::vector<int> radix;               // Stockham passes of the LZ-point DFT
    bool regs = false;                    // LZ 250 / 500 / 1000: the register-resident kernel (radix 10, 5)
    int pre_off = 0, pass_off = 0, root_off = 0, unpack_off = 0, entries = 0;
    size_t smem = 0;
};
bool mixed_plan(int64_t n, int64_t n_fft, MixedPlan* p, std::string* why);
void mixed_fill_table(const MixedPlan& p, float2* host);
cudaError_t mixed_launch(const MixedPlan& p, const float* x, int64_t batch, int n, int64_t ld_x, const float2* tab,
                         float2* X, int64_t ld_X, cudaStream_t st);

// ---- chirp-z by Bluestein (k_czt.cu) --------------------------------------
struct CztTables {
    int n = 0, m = 0, L = 0;
    uint64_t A = 0, Bh = 0;          // frac(f1/fs), frac(step/(2 fs)) in 2^-64 cycles
    float2* pre = nullptr;           // a[n] = e^{-j2pi(A n + Bh n^2)}, n < N
    float2* V = nullptr;             // FFT_L(v)/L, v[m] = e^{+j2pi Bh m^2} wrapped
    float2* post = nullptr;          // e^{-j2pi Bh k^2}, k < M
};
int czt_length(int64_t n, int64_t m);                 // power-of-two L >= N + M - 1
bool czt_supported(int64_t n, int64_t m, std::string* why);
cudaError_t czt_build_tables(const CztTables& t, const float2* tw, cudaStream_t st);
cudaError_t czt_launch(const CztTables& t, const float* x, int64_t batch, int64_t ld_x,
                       const float2* tw, float2* X, int64_t ld_X, cudaStream_t st);
// Two traces per thread (packed lanes).
bool czt_dual_ok(int L);
cudaError_t czt_launch2(const CztTables& t, const float* x, int64_t batch, int64_t ld_x,
                        const float2* tw, float2* X, int64_t ld_X, cudaStream_t st);

cudaError_t czt_pre_post_launch(const CztTables& t, cudaStream_t st);
// Segmented chirp-z for N >> M (tables of `t` built for N = seg_len): the
// segments' spectra into W [batch][segs][M], then their phase-rotated sum.
cudaError_t czt_seg_launch(const CztTables& t, const float* x, int64_t batch, int64_t n_total, int64_t ld_x,
                           int seg_len, int segs, const float2* tw, float2* W, cudaStream_t st);
cudaError_t czt_combine_launch(const float2* W, int segs, int m, int64_t batch, uint64_t A, uint64_t B,
                               int64_t seg_len, float2* X, int64_t ld_X, cudaStream_t st);

// ---- multi-pass FFT and Bluestein (k_long.cu) ------------------------------
// P = P1 x 512 points (P = N_FFT/2 for the padded FFT, L for Bluestein);
// a column pass of pruned P1-point FFTs (LZ1 nonzero inputs, R1 = P1/LZ1
// residues) and a row pass of 512-point FFTs through a workspace of P
// complex values per trace.
struct LongPlan {
    int logP = 0, logP1 = 0, LZ1 = 0, logR1 = 0;
    int logTw = 0;                   // period of the twiddle table (2P for the padded FFT)
    int64_t work_per_trace = 0;      // float2
};
bool long_fft_plan(int64_t n, int64_t n_fft, LongPlan* p, std::string* why);
bool long_czt_plan(int64_t n, int64_t m, LongPlan* p, std::string* why);
int long_fft_table_entries(const LongPlan& p);
int long_czt_table_entries(const LongPlan& p);
void long_fill_tw(const LongPlan& p, float2* host);
// work: work_traces x work_per_trace float2; the batch runs in chunks of
// work_traces traces (<= 65535).
cudaError_t long_fft_launch(const LongPlan& p, const float* x, int64_t batch, int n, int64_t ld_x,
                            const float2* block_tw_base, const float2* tw_tab, float2* work, int64_t work_traces,
                            float2* X, int64_t ld_X, cudaStream_t st);
// Tables: t.pre (N), t.V (L, in the [k1][k2] order of the row pass, scaled
// 1/L), t.post (M) and tw_tab (long_czt_table_entries, filled by the host).
cudaError_t long_czt_build_tables(const LongPlan& p, const CztTables& t, const float2* block_tw_base,
                                  float2* tw_tab, cudaStream_t st);
cudaError_t long_czt_launch(const LongPlan& p, const CztTables& t, const float2* tw_tab, const float* x,
                            int64_t batch, int64_t ld_x, const float2* block_tw_base, float2* work,
                            int64_t work_traces, float2* X, int64_t ld_X, cudaStream_t st);

// ---- chirp-z as a tensor-core product (k_gemm.cu) --------------------------
int gemm_padded_n(int64_t n);
size_t gemm_z_bytes(int64_t n, int64_t m);          // Zh | Zl, FP16 [2M][ceil64(N)] each
size_t gemm_work_bytes(int64_t batch, int64_t n);   // xh | xl | row exponents
cudaError_t gemm_build_z(int64_t n, int64_t m, uint64_t A, uint64_t B, void* z, cudaStream_t st, bool bf16 = false);
// terms 3: split FP16 (FP32-level accuracy); 1: one FP16 product; -1: one
// BF16 product (x and the BF16 Z table).  The
// split writes x's FP16 parts and row exponents into `work`
// (gemm_work_bytes(batch, n)); the product reads them.
cudaError_t gemm_split_launch(const float* x, int64_t batch, int64_t n, int64_t ld_x, int terms, void* work,
                              cudaStream_t st);
// x != null: the split runs inside the product (x read by TMA as FP32,
// 16-byte aligned rows and pitch: gemm_fused_ok); only the row exponents
// come from `work`, written by gemm_rowpow_launch.
cudaError_t gemm_mul_launch(int64_t batch, int64_t n, int64_t m, int terms, const void* z, const void* work,
                            float2* X, int64_t ld_X, unsigned* status, int sms, uint64_t timeout_ns,
                            cudaStream_t st, const int* col_pow = nullptr, const float* x = nullptr,
                            int64_t ld_x = 0);
bool gemm_fused_ok(const float* x, int64_t ld_x);
cudaError_t gemm_rowpow_launch(const float* x, int64_t batch, int64_t n, int64_t ld_x, void* work, cudaStream_t st);
// Z off the unit circle; col_pow (device, M ints): log2 of each column's scale.
cudaError_t gemm_build_z_spiral(int64_t n, int64_t m, uint64_t A, uint64_t B, double la, double lw,
                                const int* col_pow, void* z, cudaStream_t st);
cudaError_t wait_selftest_launch(unsigned* status, uint64_t timeout_ns, cudaStream_t st);

// ---- Zoom FFT (k_zoom.cu) -------------------------------------------------
struct ZoomPlan {
    int n = 0, d = 0, n_taps = 0, K = 0, lout = 0;
    int rs = 0;      // polyphase row stride (floats, odd)
    uint64_t Cn = 0; // frac(f_N / fs) in 2^-64 cycles
    int threads = 0;
    size_t smem = 0;
    bool dual = false;   // two traces per CTA (packed lanes)
    size_t smem2 = 0;
    bool big = false;    // FIR kernel + pruned cluster FFT (zoom_big_*)
    FftPlan fft;         // the K-point FFT of the big path
};
bool zoom_plan(int64_t n, int64_t d, int64_t n_taps, int64_t n_fft, double fs, double f1,
               double f2, ZoomPlan* p, std::string* why);
// Large Zoom FFTs: FIR-decimate into `work` ([batch][fft.LZ] float2), then
// the pruned cluster FFT.
bool zoom_big_plan(int64_t batch, int64_t n, int64_t d, int64_t n_taps, int64_t n_fft, double fs, double f1,
                   double f2, ZoomPlan* p, std::string* why);
cudaError_t zoom_big_launch(const ZoomPlan& p, const float* x, int64_t batch, int64_t ld_x, const float* taps,
                            float2* work, const float2* tw, const float2* tab, float2* X, int64_t ld_X,
                            cudaStream_t st);
cudaError_t zoom_launch(const ZoomPlan& p, const float* x, int64_t batch, int64_t ld_x,
                        const float* taps, const float2* tw, float2* X, int64_t ld_X, cudaStream_t st,
                        int lanes);

// ---- ragged batches (ragged.cu drives these) -------------------------------
// Persistent chirp-z over a work queue (k_czt.cu): units of max(1, 8192/L)
// traces of one Bluestein length L, largest L first; items[].tab_off is the offset of
// the trace's FFT(v)/L in vpool (one per distinct (N, M, B)).
struct CztUnit {
    int L;          // Bluestein length of the unit's traces
    int first;      // first item (index into the item array)
    int count;      // traces in the unit (<= 16384 / L)
    int pad;
};
// Persistent padded FFT over a work queue (k_fft.cu): mode 0 units hold
// 512/(R/2 LZ/16) whole traces (H <= 16384), mode 1 units `count` residue
// pairs g0 .. of one trace (item), mode 2 units one trace through a per-CTA
// workspace; tab is the (LZ, R) plan's generic table.
struct FftUnit {
    const float2* tab;
    int LZ, logR;
    int item, count, g0, mode;
};
size_t fft_queue_smem();
// ws: ctas x ws_per_cta complex values (mode 2 units: ws_per_cta >= H); the
// grid has exactly `ctas` CTAs (each owns one workspace slot)
cudaError_t fft_queue_launch(const RaggedItem* items, const FftUnit* units, int nunits, unsigned* counter,
                             const float* x_pool, const float2* btw, float2* X_pool, float2* ws, int64_t ws_per_cta,
                             int ctas, cudaStream_t st);
// Persistent Zoom FFT over a work queue (k_zoom.cu): a unit is up to F
// traces of one K <= 16384 (F <= 1024/(K/16)), trace f in the `slice`-byte
// shared-memory slice f; thread groups without a trace use the FFT area at
// byte `scratch` (valid when count < 1024/(K/16)).
struct ZoomUnit {
    int K, first, count, F;
    int slice, scratch;
};
int zoom_queue_groups(int K);
cudaError_t zoom_queue_launch(const RaggedItem* items, const ZoomUnit* units, int nunits, unsigned* counter,
                              size_t smem, const float* x_pool, const float* taps_pool, const float2* tw,
                              float2* X_pool, int ctas, cudaStream_t st);
size_t czt_queue_smem();
int czt_queue_unit_traces(int L);
cudaError_t czt_vpool_build(int L, const RaggedItem* keys, int64_t count, float2* vpool, const float2* tw_base,
                            cudaStream_t st);
cudaError_t czt_queue_launch(const RaggedItem* items, const CztUnit* units, int nunits, unsigned* counter,
                             const float* x_pool, const float2* vpool, const float2* tw_base, const float2* tw32_base,
                             float2* X_pool, int ctas, cudaStream_t st);
cudaError_t czt_ragged_tables(int L, const RaggedItem* items, int64_t count, float2* tables, const float2* tw,
                              cudaStream_t st);
cudaError_t czt_ragged_launch(int L, const RaggedItem* items, int64_t count, const float* x_pool,
                              const float2* tables, const float2* tw, float2* X_pool, cudaStream_t st);
int zoom_rows(int64_t lout, int64_t n_taps, int64_t d);
size_t zoom_smem_for(int n_taps, int d, int rs, int K);
int fir_rows(int64_t n_taps, int64_t d);
size_t fir_smem_for(int n_taps, int d);
int fir_chunk();
// lo4: every trace of the class has L_out <= K/4 (the kernel's sparse first FFT pass)
cudaError_t zoom_ragged_launch(int K, const RaggedItem* items, int64_t count, size_t smem, const float* x_pool,
                               const float* taps_pool, const float2* tw, float2* X_pool, cudaStream_t st,
                               bool lo4 = false);
cudaError_t zoom_fir_ragged_launch(const RaggedItem* items, int64_t count, int chunks_max, size_t smem,
                                   const float* x_pool, const float* taps_pool, float2* work, cudaStream_t st);

}  // namespace spec
