/*
 * spec.h -- C-ABI of the batched spectral-estimation library for sampled
 * THz-TDS traces (zero-padded FFT, chirp-z transform, Zoom FFT), after
 * García-Devesa, Báez-Chorro and Vidal, "Comparison of computing efficiency
 * among FFT, CZT and Zoom FFT in THz-TDS", arXiv 2108.03948.
 *
 * Data layout shared by every transform
 *   x   real float32 traces, row-major [batch][ld_x]; the first n samples of a
 *       row are the trace x[n] = x(n T_s), T_s = 1/fs (Section 2.1, Eq. 1).
 *   X   complex64 spectra, row-major [batch][ld_X], each element two floats
 *       (re, im) interleaved; ld_X counts complex elements.
 *   x and X may be device pointers (async on `stream`, no host sync) or host
 *   pointers (pageable or pinned): host buffers are staged through
 *   library-owned device memory in chunks of traces, the upload of one chunk,
 *   the transform of the previous one (on `stream`) and the download of the
 *   one before overlapping (fully so with pinned memory), and the call
 *   returns once X holds the result.
 *   The caller owns x, X and the taps; the library owns only what sits in the
 *   context (tables, caches, staging buffers).
 *   `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *
 * Errors
 *   Every argument is validated before any launch; a bad one returns
 *   SPEC_EINVAL and touches no memory.  Nothing aborts and nothing throws
 *   across this boundary; spec_last_error() gives a one-line reason.
 *   One context per host thread.
 */
#ifndef SPEC_H
#define SPEC_H

#include <stdint.h>

#if defined(__GNUC__)
#define SPEC_API __attribute__((visibility("default")))
#else
#define SPEC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPEC_OK = 0,
    SPEC_EINVAL = 1,        /* bad argument (checked before any launch)        */
    SPEC_ENOMEM = 2,        /* device or host allocation failed                 */
    SPEC_ECUDA = 3,         /* a CUDA runtime call failed                       */
    SPEC_EUNSUPPORTED = 4,  /* valid arguments beyond the library's size limits */
    SPEC_ETIMEOUT = 5       /* a bounded device-side wait gave up               */
} spec_status;

/* How spec_czt evaluates the chirp-z transform.
 *   SPEC_CZT_AUTO          the library picks by measurement: the first call
 *                          with a given (N, M, batch rounded up to a power of
 *                          two) runs Bluestein and SPEC_CZT_GEMM_F16X3 on a
 *                          probe batch of synthetic traces on the device,
 *                          admits the product only if its spectra agree with
 *                          Bluestein's to 1e-5 relative L2 each, and keeps
 *                          the faster (synchronises the stream; the decision
 *                          is remembered in the context and, if the
 *                          environment variable SPEC_AUTOTUNE_CACHE names a
 *                          file when the context is created, in that file --
 *                          see spec_czt_auto_mode).
 *   SPEC_CZT_BLUESTEIN     FP32 Bluestein: chirp, FFT convolution, chirp
 *                          (Section 2.3, Eq. 13-15).
 *   SPEC_CZT_GEMM_F16X3    Eq. 11 as the product x Z^T, Z[k][n] = z_k^{-n},
 *                          on the tensor cores: x (per-row power-of-two
 *                          scale) and Z each split into two FP16 parts, three
 *                          products accumulated in FP32.  Relative error a
 *                          few 1e-7, like the FP32 path.  The paper has no
 *                          counterpart (it uses Bluestein only).
 *   SPEC_CZT_GEMM_F16X1    the same with one FP16 product: relative error
 *                          about 1e-3 (below the 1e-5 bar; for screening).
 *   SPEC_CZT_GEMM_BF16X1   one BF16 product (x and Z rounded once to BF16,
 *                          FP32 accumulation): the single-term BF16 error,
 *                          about 3e-3 relative (below the 1e-5 bar; reported
 *                          beside the split form, not an accurate mode).
 * The GEMM modes cache Z (2 x 2M x ceil64(N) FP16) per (N, M, f1/fs,
 * step/fs) and use a workspace of 4 bytes per input sample.             */
typedef enum {
    SPEC_CZT_AUTO = 0,
    SPEC_CZT_BLUESTEIN = 1,
    SPEC_CZT_GEMM_F16X3 = 2,
    SPEC_CZT_GEMM_F16X1 = 3,
    SPEC_CZT_GEMM_BF16X1 = 4
} spec_czt_mode;

typedef struct spec_ctx spec_ctx;

/* Create a context bound to CUDA device `device`.  Allocates nothing large;
 * tables are built on first use and cached.  Returns SPEC_EINVAL for a bad
 * device index or a NULL out-pointer, SPEC_ECUDA if the device cannot be
 * used.  On failure *ctx is set to NULL. */
SPEC_API spec_status spec_ctx_create(spec_ctx** ctx, int device);

/* Free every device buffer the context owns.  Synchronises the device.
 * NULL is accepted. */
SPEC_API void spec_ctx_destroy(spec_ctx* ctx);

/* One-line reason for the last non-OK status returned on this context
 * (empty string if none).  Valid until the next call on the context.
 * A NULL context gives the reason of the last failed spec_ctx_create. */
SPEC_API const char* spec_last_error(const spec_ctx* ctx);

/* Wait for `stream` and report any deferred device-side error: SPEC_ECUDA
 * for a CUDA error, SPEC_ETIMEOUT if a bounded device wait gave up (the
 * tensor-core kernels bound every wait on their pipeline barriers; a wait
 * that gives up leaves that call's output incomplete).  Reading the status
 * clears it. */
SPEC_API spec_status spec_ctx_check(spec_ctx* ctx, void* stream);

/* Measure the device's FP32 FMA throughput (TFLOP/s) with a packed-FMA
 * microbenchmark (a few ms; synchronises `stream`).  The denominator of the
 * ALU roofline reported for the FP32 transforms.  No counterpart in the
 * paper. */
SPEC_API spec_status spec_measure_fp32_peak(spec_ctx* ctx, double* tflops, void* stream);

/* Self-test of the bounded-wait machinery: launches one CTA that waits on
 * a barrier nothing will complete, with a limit of `timeout_us`
 * microseconds (1 .. 10^6).  The next spec_ctx_check on `stream` must then
 * return SPEC_ETIMEOUT.  No counterpart in the paper. */
SPEC_API spec_status spec_selftest_wait_timeout(spec_ctx* ctx, int64_t timeout_us, void* stream);

/*
 * Kernel variants.  spec_fft, spec_czt (Bluestein) and spec_zoom have
 * several kernels for one shape (two traces or residues per thread as packed
 * lanes or one; for the FFT also a kernel compiled for the shape, and a
 * cluster kernel for long traces).  The first call with a device-resident
 * batch of a given shape runs each variant three times on the call's own
 * buffers, keeps the fastest for that shape (every later call, and every
 * chunk of a host-buffer call, runs the same arithmetic) and so synchronises
 * `stream` once; the choice is also stored in the SPEC_AUTOTUNE_CACHE file
 * (see spec_czt_auto_mode).  During stream capture nothing is timed and the
 * first variant runs.  SPEC_LANES=1 or 2 in the environment at context
 * creation pins the lanes instead.
 */

/*
 * Zero-padded FFT of real traces (Section 2.1, Eq. 2 with the forward sign
 * e^{-j 2 pi k n / N_FFT}; the zero-padding paragraph; resolution
 * Delta f = fs/N_FFT, Eq. 3):
 *
 *     X[b][k] = sum_{n<N} x[b][n] e^{-j 2 pi k n / N_FFT},  k = 0 .. N_FFT/2
 *
 * The input is real, so the N_FFT/2 + 1 non-redundant bins are written
 * (unnormalised); bin k is frequency k fs / N_FFT.
 *   n      samples per trace, 1 <= n <= n_fft (no truncation)
 *   n_fft  padded length, 1 <= n_fft <= 2^24; powers of two run the padded
 *          FFT, any other length (e.g. N_FFT = fs / Delta f for the
 *          resolution of Eq. 3-5) the chirp-z on the DFT grid (f1 = 0,
 *          step fs / N_FFT, N_FFT/2 + 1 points), which gives the same bins
 *   fs     sampling frequency (> 0); defines the bin grid only
 *   ld_x >= n, ld_X >= n_fft/2 + 1; x and X must not overlap.
 */
SPEC_API spec_status spec_fft(spec_ctx* ctx, const float* x, int64_t batch, int64_t n,
                     int64_t ld_x, double fs, int64_t n_fft,
                     float* X, int64_t ld_X, void* stream);

/*
 * Chirp-z transform on the unit circle (Section 2.3, Eq. 11 with Eq. 16-23,
 * A_0 = W_0 = 1):
 *
 *     X[b][k] = sum_{n<N} x[b][n] A^{-n} W^{k n},  k = 0 .. M-1,
 *     A = e^{j 2 pi f1/fs},  W = e^{-j 2 pi (f2 - f1)/(fs (M - 1))}
 *
 * i.e. the trace's spectrum at f_k = f1 + k (f2 - f1)/(M - 1): both band
 * edges are bins (the (N_CZT - 1) of Eq. 18).  M = 1 gives the single bin
 * at f1.  f2 < f1 is allowed (descending grid).  To get the paper's Eq. 24
 * spacing (f2 - f1)/M pass f2' = f1 + (f2 - f1)(M - 1)/M.
 * Unnormalised.  Bluestein form: X[k] = W^{k^2/2} [(x A^{-n} W^{n^2/2})
 * (*) W^{-n^2/2}] (Eq. 13-15) over a power-of-two length L >= N + M - 1.
 *   n >= 1, m >= 1, fs > 0, finite f1 and f2; ld_x >= n, ld_X >= m.
 *   mode: see spec_czt_mode.
 */
SPEC_API spec_status spec_czt(spec_ctx* ctx, const float* x, int64_t batch, int64_t n,
                     int64_t ld_x, double fs, double f1, double f2, int64_t m,
                     int mode, float* X, int64_t ld_X, void* stream);

/*
 * Chirp-z off the unit circle (Section 2.3, Eq. 11 with Eq. 16-17, A_0 and
 * W_0 free):
 *
 *     X[b][k] = sum_{n<N} x[b][n] A^{-n} W^{k n},  k = 0 .. M-1,
 *     A = a0 e^{j 2 pi f1/fs},  W = w0 e^{-j 2 pi (f2 - f1)/(fs (M - 1))}
 *
 * i.e. the z-transform on the spiral z_k = A W^{-k} (radius a0 w0^{-k});
 * a0 = w0 = 1 gives spec_czt's bins.  Evaluated as the split-FP16
 * tensor-core product (SPEC_CZT_GEMM_F16X3) with Z's column k scaled by a
 * power of two, so that each bin is a direct dot product (Bluestein's
 * factors w0^{+-n^2/2} leave FP32 range for all but the mildest spirals).
 *   a0, w0 > 0; SPEC_EUNSUPPORTED when |z_k|^{-n} exceeds 2^100 for some
 *   k, n, or when Z (2 x 2M x ceil64(N) FP16) exceeds 2 GiB.  Other
 *   arguments as spec_czt.
 */
SPEC_API spec_status spec_czt_spiral(spec_ctx* ctx, const float* x, int64_t batch, int64_t n,
                            int64_t ld_x, double fs, double f1, double f2, int64_t m,
                            double a0, double w0, float* X, int64_t ld_X, void* stream);

/*
 * Zoom FFT (Section 2.2, Eq. 6-10): the spectrum around the band centre
 * f_N = (f1 + f2)/2 (Eq. 6) at the FFT's spacing fs/N_FFT:
 *
 *     y[n] = x[n] e^{-j 2 pi f_N n / fs}                  (Eq. 7, down-shift)
 *     u[m] = sum_{k<L_h} h[k] y[m D - k],  y = 0 outside [0, N)   (Eq. 8-10)
 *            m = 0 .. L_out - 1,  L_out = ceil((N + L_h - 1)/D)
 *     U[j] = sum_m u[m] e^{-j 2 pi j m / K},  K = N_FFT / D       (Eq. 9)
 *     X[b][i] = U[(i - K/2) mod K],  i = 0 .. K-1   (ascending frequency:
 *               bin i is f_N + (i - K/2) fs / N_FFT)
 *
 *   taps   h[0 .. n_taps-1], float32, device or host pointer, used as given
 *          (spec_design_lowpass makes the Hamming low-pass used by the
 *          benchmarks)
 *   d      decimation D >= 1, n_fft % d == 0, K = n_fft/d a power of two
 *   L_out <= K is required (the kept samples must fit the K-point FFT).
 *   ld_x >= n, ld_X >= K.
 */
SPEC_API spec_status spec_zoom(spec_ctx* ctx, const float* x, int64_t batch, int64_t n,
                      int64_t ld_x, double fs, double f1, double f2, int64_t d,
                      const float* taps, int64_t n_taps, int64_t n_fft,
                      float* X, int64_t ld_X, void* stream);

/*
 * spec_czt without any device allocation (the paper has no counterpart;
 * this is a deployment variant of spec_czt).
 *
 * For callers that cannot allocate device memory: code whose device memory
 * is owned by another allocator (a framework's caching pool that has
 * reserved it), real-time loops that must not call cudaMalloc (it may
 * synchronise the device and has unbounded latency), plug-ins handed
 * buffers but no allocator.  It needs no context.
 *
 * Same transform, arguments and accuracy as spec_czt in Bluestein mode,
 * except:
 *   - x and X must be device pointers (SPEC_EINVAL otherwise);
 *   - N + M - 1 <= 8192, else SPEC_EUNSUPPORTED before any launch;
 *   - working memory is one file-scope device array of about 320 KiB (FFT
 *     twiddles, chirp tables and the chirp kernel's spectrum) that every
 *     GPU loading the library keeps until the process exits;
 *   - the first call on each device (the current device) fetches the
 *     array's device address, fills its twiddles and synchronises `stream`;
 *     make that first call before any stream capture;
 *   - every call rewrites the chirp tables in that shared array, so calls
 *     that overlap on the GPU (e.g. on two streams) race: order them on one
 *     stream;
 *   - the set-up belongs to the device's CUDA context: do not use this entry
 *     point across a cudaDeviceReset in the same process (the array is
 *     reloaded and its twiddles are lost while the set-up is remembered).
 * Returns SPEC_ECUDA if a CUDA call fails.
 */
SPEC_API spec_status spec_czt_static(const float* x, int64_t batch, int64_t n, int64_t ld_x,
                                     double fs, double f1, double f2, int64_t m,
                                     float* X, int64_t ld_X, void* stream);

/*
 * The explicit mode SPEC_CZT_AUTO stands for at (batch, n, m): taken from the
 * context, or from the SPEC_AUTOTUNE_CACHE file read at context creation, or
 * measured now on a device probe batch (synchronises `stream`).  This is the
 * autotuner the paper's cost comparison of Section 2.3 (after Eq. 25) and
 * Section 4 motivates: the faster exact evaluation of Eq. 11 per shape.
 * *mode receives SPEC_CZT_BLUESTEIN or SPEC_CZT_GEMM_F16X3; a following
 * spec_czt call with that mode computes bit for bit what SPEC_CZT_AUTO does.
 */
SPEC_API spec_status spec_czt_auto_mode(spec_ctx* ctx, int64_t batch, int64_t n, double fs, double f1, double f2,
                                        int64_t m, int* mode, void* stream);

/*
 * The decision cache file (host only, no device needed; no counterpart in
 * the paper).  One JSON object {"format": "spec-autotune-1", "device": tag,
 * "entries": {key: value}}; keys and values use only letters, digits and
 * "_.:=| -".  spec_tune_cache_store adds or replaces one entry, keeping the
 * file's other entries only if they were written for the same device tag
 * and format (a file from another device or format is replaced), through a
 * temporary file and a rename; returns 0, or -1 if the file cannot be
 * written.  spec_tune_cache_lookup returns 1 and copies the value (truncated
 * to cap - 1 characters) if the file exists, parses, has this device tag and
 * format, and holds the key; else 0.
 */
SPEC_API int spec_tune_cache_store(const char* path, const char* device, const char* key, const char* value);
SPEC_API int spec_tune_cache_lookup(const char* path, const char* device, const char* key, char* value, int cap);

/*
 * Ragged batches: many traces, each with its own length, band, point count,
 * decimation and taps, in one call.  Each descriptor is one independent
 * spec_fft / spec_czt / spec_zoom problem on one trace (the paper's three
 * transforms, Sections 2.1-2.3, with the conventions documented above):
 *   trace   x_pool[x_off .. x_off + n)
 *   output  X_pool + out_off (complex elements): n_fft/2 + 1 bins (FFT),
 *           m bins (CZT) or n_fft/d bins (Zoom), in the orders above
 *   kind    SPEC_KIND_FFT uses n, n_fft; SPEC_KIND_CZT uses n, f1, f2, m;
 *           SPEC_KIND_ZOOM uses n, f1, f2, d, n_fft and the taps
 *           taps_pool[taps_off .. taps_off + n_taps).
 * fs is shared by the batch.  The pools are device pointers; the descriptor
 * array is host memory and is copied.  Outputs of different descriptors
 * must not overlap (not checked).
 * The first call with a descriptor list synchronises `stream`, builds a plan
 * and caches it in the context: per kind one persistent launch over a work
 * queue of units (a few traces of one shape, or part of one long trace),
 * largest first, popped by one CTA per SM; traces beyond the queue kernels'
 * sizes (padded-FFT residue FFTs above 4096 points, Zoom N_FFT/d above
 * 16384) run as per-shape launches in the same graph; the alternatives a
 * plan admits are timed and the fastest kept.  A repeated call with
 * identical descriptors and pools is one graph launch, asynchronous on
 * `stream`.  Every descriptor is validated before anything
 * runs (SPEC_EINVAL / SPEC_EUNSUPPORTED with the descriptor's index in
 * spec_last_error).
 */
typedef enum { SPEC_KIND_FFT = 0, SPEC_KIND_CZT = 1, SPEC_KIND_ZOOM = 2 } spec_kind;

typedef struct {
    int64_t x_off;      /* first sample in x_pool (floats)              */
    int64_t n;          /* samples                                      */
    int64_t out_off;    /* first bin in X_pool (complex elements)       */
    double f1, f2;      /* band (CZT, Zoom)                             */
    int64_t n_fft;      /* padded length (FFT, Zoom)                    */
    int64_t m;          /* CZT points                                   */
    int64_t d;          /* Zoom decimation                              */
    int64_t taps_off;   /* first tap in taps_pool (Zoom)                */
    int64_t n_taps;     /* taps (Zoom)                                  */
} spec_desc;

SPEC_API spec_status spec_ragged(spec_ctx* ctx, int kind, const spec_desc* descs, int64_t count, double fs,
                                 const float* x_pool, const float* taps_pool, float* X_pool, void* stream);

/* Kernel launches one replay of the cached plan for these descriptors makes
 * (the work-queue launch if the plan uses it, one per remaining class of
 * traces, plus one FIR launch for Zoom FFTs too large for one CTA), or -1 if
 * the context holds no such plan.  Library bookkeeping; the paper has no
 * counterpart.  (SPEC_RAGGED_QUEUE=1 or 0 in the environment when a context
 * is created makes its plans always, or never, use the work queue.) */
SPEC_API int64_t spec_ragged_launches(const spec_ctx* ctx, int kind, const spec_desc* descs, int64_t count,
                                      double fs);

/*
 * How the cached plan for these descriptors runs (no counterpart in the
 * paper; host only, no device work): returns 1 if its graph launches the
 * persistent work queue, 0 if the per-shape launches were faster when the
 * plan was built (both forms are timed then; their times in microseconds go
 * to *t_queue_us and *t_classes_us, 0 where the plan has no queue), -1 if
 * the context holds no plan for these descriptors.  Either pointer may be
 * NULL.
 */
SPEC_API int spec_ragged_plan_info(const spec_ctx* ctx, int kind, const spec_desc* descs, int64_t count, double fs,
                                   float* t_queue_us, float* t_classes_us);

/* ---- host-only helpers (pure functions, no CUDA calls) ----------------- */

/* Zeros to append to an N_FFT-sample record so that its bin spacing shrinks
 * by `delta` (Section 2.1, Eq. 4-5: Delta = fs/N_FFT - fs/(N_FFT + x),
 * x = fs N_FFT/(fs - Delta N_FFT) - N_FFT), rounded up to the smallest
 * integer that reaches delta.  Returns -1 if fs <= 0, n_fft <= 0, delta < 0
 * or delta >= fs/n_fft. */
SPEC_API int64_t spec_zeros_for_delta(double fs, int64_t n_fft, double delta);

/* CZT points giving the FFT's spacing over [f1, f2] (Section 2.3, Eq. 25:
 * N_CZT = (f2 - f1)/fs N_FFT), rounded up; at least 1.  -1 for fs <= 0 or
 * n_fft <= 0. */
SPEC_API int64_t spec_m_for_resolution(double fs, double f1, double f2, int64_t n_fft);

/* Low-pass FIR for the Zoom FFT decimator (Section 2.2, Eq. 8 realised as a
 * finite filter): Hamming-windowed sinc with cutoff fs/(2D),
 * h[k] = (0.54 - 0.46 cos(2 pi k/(L_h - 1))) sinc((k - (L_h - 1)/2)/D)/D,
 * scaled so that sum h = D.  Writes n_taps floats to host memory `taps`.
 * SPEC_EINVAL for n_taps < 1, d < 1 or taps == NULL. */
SPEC_API spec_status spec_design_lowpass(float* taps, int64_t n_taps, int64_t d);

#ifdef __cplusplus
}
#endif

#endif /* SPEC_H */
