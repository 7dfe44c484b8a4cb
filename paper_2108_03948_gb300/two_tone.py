"""Two-tone resolvability: the experiment of Section 3.1 on the GPU.

Two unit sines (zero phase) at f_a and f_a + delta, 128 samples at
fs = 8 kHz.  The chirp-z looks at 100 - 1000 Hz with the paper's plotting
resolution of 7.03 Hz (the grid of Eq. 24: M = 128 points spaced
(f2 - f1)/M, i.e. f2' = f1 + (f2 - f1)(M - 1)/M under the M - 1 convention);
the zero-padded FFT is taken at the same plotting resolution,
N_FFT = round(fs / 7.03 Hz) = 1138 (any length runs).  For each separation
delta the spectrum's two largest peaks near the tones and the lowest point
between them give the dip ratio (dip / smaller peak); the tones count as
resolved when that ratio is below 1/sqrt(2) (a 3 dB dip).  The paper's
claim: the chirp-z does not resolve tones earlier than the FFT with the same
plotting resolution -- both are bounded by the 128-sample window
(fs / N = 62.5 Hz).

Usage: python -m paper_2108_03948_gb300.two_tone
Prints: delta (Hz), dip ratio of the FFT, dip ratio of the CZT.
"""
from __future__ import annotations

import sys

import numpy as np

from . import spec


def dip_ratio(freqs: np.ndarray, mag: np.ndarray, fa: float, fb: float) -> float:
    """Lowest magnitude between the peaks nearest fa and fb over the smaller
    peak (1.0 if the two nearest maxima coincide)."""
    ia = int(np.argmin(np.abs(freqs - fa)))
    ib = int(np.argmin(np.abs(freqs - fb)))
    # climb to the local maxima around each tone
    def climb(i):
        while 0 < i < len(mag) - 1 and (mag[i - 1] > mag[i] or mag[i + 1] > mag[i]):
            i = i - 1 if mag[i - 1] > mag[i + 1] else i + 1
        return i
    pa, pb = climb(ia), climb(ib)
    if pa == pb:
        return 1.0
    lo, hi = min(pa, pb), max(pa, pb)
    return float(mag[lo:hi + 1].min() / min(mag[pa], mag[pb]))


def main(argv=None) -> int:
    import torch
    fs, n = 8000.0, 128
    f1, f2, m = 100.0, 1000.0, 128
    f2p = f1 + (f2 - f1) * (m - 1) / m                 # the Eq. 24 grid, step (f2 - f1)/M
    n_fft = int(round(fs / ((f2 - f1) / m)))           # same plotting resolution, 1138
    fa = 400.0
    deltas = np.arange(20.0, 141.0, 5.0)
    t = np.arange(n) / fs
    x = np.stack([np.sin(2 * np.pi * fa * t) + np.sin(2 * np.pi * (fa + d) * t) for d in deltas]).astype(np.float32)
    ctx = spec.Context(0)
    xd = torch.from_numpy(x).cuda()
    X = spec.spec_fft(ctx, xd, fs, n_fft).abs().cpu().numpy()
    Z = spec.spec_czt(ctx, xd, fs, f1, f2p, m).abs().cpu().numpy()
    ctx.close()
    ffreq = np.arange(n_fft // 2 + 1) * fs / n_fft
    cfreq = f1 + np.arange(m) * (f2p - f1) / (m - 1)
    print(f"# plotting resolution: FFT {fs / n_fft:.2f} Hz (N_FFT = {n_fft}), CZT {(f2p - f1) / (m - 1):.2f} Hz; "
          f"window resolution fs/N = {fs / n:.1f} Hz")
    print("delta_Hz fft_dip czt_dip")
    first = {"fft": None, "czt": None}
    for i, d in enumerate(deltas):
        rf = dip_ratio(ffreq, X[i], fa, fa + d)
        rc = dip_ratio(cfreq, Z[i], fa, fa + d)
        for k, r in (("fft", rf), ("czt", rc)):
            if first[k] is None and r < 2 ** -0.5:
                first[k] = d
        print(f"{d:.0f} {rf:.3f} {rc:.3f}")
    print(f"# first separation with a 3 dB dip: FFT {first['fft']} Hz, CZT {first['czt']} Hz")
    return 0


if __name__ == "__main__":
    sys.exit(main())
