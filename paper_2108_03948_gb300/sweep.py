"""Resolution sweep: the timing experiment of Section 4 (Fig. 11) on the GPU.

The paper runs each method 10000 times per spectral resolution, from
Delta f = 20 GHz down in 0.5 GHz steps, on THz-TDS traces of N = 500 samples
at T_s = 100 fs (fs = 10 THz), and plots each method's time relative to its
first point.  Here the 10000 runs are one batch of 10000 synthetic traces of
that shape (one launch sequence per method), timed with CUDA events.

Per resolution Delta f:
  FFT   N_FFT = ceil(fs / Delta f) (Eq. 3; the zeros of Eq. 5 are N_FFT - N),
        any length (powers of two run the padded FFT, even lengths whose half
        has only the factors 2, 3, 5, 7 the mixed-radix padded FFT, others the
        chirp-z on the DFT grid);
  CZT   the band f1 .. f2 at M = ceil((f2 - f1) N_FFT / fs) points (Eq. 25);
  Zoom  the same band, decimation D the largest power of two with
        fs / D >= 1.25 (f2 - f1), K = N_FFT / D rounded up to a power of two
        (so its Delta f = fs / (K D) is at most the requested one).
The band is not stated in the paper; 0.1 - 3.0 THz (the usable THz-TDS band
of such traces) is used.

Usage: python -m paper_2108_03948_gb300.sweep [--traces 10000] [--steps 40]
Prints one line per resolution: Delta f, the sizes and the times (us) of the
three methods, and each time relative to the first resolution.
"""
from __future__ import annotations

import argparse
import math
import sys

import numpy as np

from . import spec, synth


def _time(f, reps: int, flush) -> float:
    import torch
    for _ in range(2):
        f()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        f()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) * 1e3)
    return float(np.median(ts))


def zoom_decimation(fs: float, f1: float, f2: float) -> int:
    """The largest power of two D with fs / D >= 1.25 (f2 - f1): the decimated
    rate still covers the band with a 25% guard."""
    d = 1
    while fs / (2 * d) >= 1.25 * (f2 - f1):
        d *= 2
    return d


def sizes(fs: float, n: int, f1: float, f2: float, df: float, d: int, n_taps: int = 63):
    """(N_FFT, M, K) of one resolution Delta f: N_FFT = ceil(fs / Delta f)
    (Eq. 3, never below N), M = ceil((f2 - f1) N_FFT / fs) (Eq. 25), and the
    Zoom FFT's K = N_FFT / D rounded up to a power of two and large enough for
    the ceil((N + L_h - 1) / D) decimated samples."""
    n_fft = max(n, math.ceil(fs / df))
    m = spec.spec_m_for_resolution(fs, f1, f2, n_fft)
    k = 1 << max(0, math.ceil(math.log2(n_fft / d)))
    while (n + n_taps - 1 + d - 1) // d > k:
        k *= 2
    return n_fft, m, k


def main(argv=None) -> int:
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--traces", type=int, default=10000)
    ap.add_argument("--steps", type=int, default=40, help="resolutions 20 GHz - 0.5 GHz i, i < steps")
    ap.add_argument("--reps", type=int, default=10)
    args = ap.parse_args(argv)

    fs, n = 10e12, 500
    f1, f2 = 0.1e12, 3.0e12
    rng = np.random.default_rng(2108)
    ps = 1e-12
    x = np.stack([synth.trace(n, fs, rng.uniform(0.2, 0.35) * ps, rng.uniform(10, 20) * ps,
                              [(rng.uniform(2, 10) * ps, rng.uniform(0.1, 0.5))], rng.uniform(40, 70), rng)
                  for _ in range(args.traces)]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    ctx = spec.Context(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    D = zoom_decimation(fs, f1, f2)
    taps = torch.from_numpy(spec.spec_design_lowpass(63, D)).cuda()
    first = None
    print("delta_f_GHz n_fft fft_us czt_m czt_us zoom_D zoom_K zoom_us fft_rel czt_rel zoom_rel")
    for i in range(args.steps):
        df = 20e9 - 0.5e9 * i
        n_fft, m, K = sizes(fs, n, f1, f2, df, D)
        X = torch.empty((args.traces, n_fft // 2 + 1), dtype=torch.complex64, device="cuda")
        Z = torch.empty((args.traces, m), dtype=torch.complex64, device="cuda")
        U = torch.empty((args.traces, K), dtype=torch.complex64, device="cuda")
        t_fft = _time(lambda: spec.spec_fft(ctx, xd, fs, n_fft, out=X), args.reps, flush)
        t_czt = _time(lambda: spec.spec_czt(ctx, xd, fs, f1, f2, m, out=Z), args.reps, flush)
        t_zoom = _time(lambda: spec.spec_zoom(ctx, xd, fs, f1, f2, D, taps, K * D, out=U), args.reps, flush)
        if first is None:
            first = (t_fft, t_czt, t_zoom)
        print(f"{df / 1e9:.1f} {n_fft} {t_fft:.1f} {m} {t_czt:.1f} {D} {K} {t_zoom:.1f} "
              f"{t_fft / first[0]:.2f} {t_czt / first[1]:.2f} {t_zoom / first[2]:.2f}", flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
