"""FP64 CPU oracle for the three spectral transforms of García-Devesa, Báez-Chorro
and Vidal, "Comparison of computing efficiency among FFT, CZT and Zoom FFT in
THz-TDS" (arXiv 2108.03948).

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline / reference legs of
``bench.py``; nothing on the product path may import or call it.  It shares no
code with the CUDA library: it reads float32 (or float64) arrays and evaluates
each transform by its definition, in float64, with numpy's BLAS matmul as the
only library step.  No blocking, fusion or reordering beyond what the cited
definition states.

Conventions (each a reading of the paper where it is silent or garbled):

* DFT sign.  Section 2.1, Eq. 2 writes ``W^{-kn}`` with ``W = e^{-j2pi/N}``,
  which is the inverse-DFT sign; the CZT reduction stated after Eq. 11
  (``A = 1, W = e^{-j2pi/N}`` with ``W^{kn}``) fixes the forward sign
  ``e^{-j2pi kn/N}``, used throughout.
* FFT output.  The input is real, so the ``N_FFT/2 + 1`` non-redundant bins are
  returned; zero padding appends zeros after the ``N`` samples (Section 2.1).
* CZT contour.  Eq. 16-23 with ``A_0 = W_0 = 1`` (unit circle): start angle
  ``theta_0 = 2pi f1/fs`` (Eq. 19, the start of the band) and step
  ``phi_0 = 2pi (f2 - f1) / (fs (M - 1))`` (Eq. 18); Eq. 20-21 print the two
  symbols swapped.  Both band edges are bins; ``M = 1`` has step 0.
* Zoom FFT mix.  Eq. 7 is garbled (no ``n``, no ``2pi``); the down-shift that
  moves the band centre ``f_N`` (Eq. 6) to DC is ``y[n] = x[n] e^{-j2pi f_N n/fs}``.
* Zoom FFT filter.  Eq. 10 is a causal FIR with zero initial state, taps
  ``k = 0 .. L_h - 1`` (the printed upper limit ``N - 1`` is the signal length);
  the full convolution is kept, so ``m = 0 .. ceil((N + L_h - 1)/D) - 1``.
* Zoom FFT length and order.  ``K = N_FFT / D`` points (the length ``L_D = L/D``
  after Eq. 9, so that the bin spacing equals the FFT's ``fs/N_FFT``); the
  output is in ascending frequency: bin ``i`` is ``f_N + (i - K/2) fs/N_FFT``.
* Phases are reduced to cycles before the trigonometric call: integer products
  ``k n`` are taken modulo the transform length exactly (int64), and real
  products ``a n`` keep only their fractional part.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "fft_padded", "fft_padded_bins",
    "czt", "czt_bins", "czt_grid", "czt_spiral", "czt_spiral_bins",
    "zoom", "zoom_bins", "zoom_grid", "zoom_lout",
    "fft_resolution", "zeros_for_delta", "czt_step", "czt_resolution_eq24",
    "m_for_resolution", "design_lowpass",
]

# Column chunk for the explicit DFT matrices: keeps each (N x chunk) float64
# matrix near 64 MB whatever the transform size.
_CHUNK_ELEMS = 1 << 23


def _as_batch(x) -> np.ndarray:
    a = np.asarray(x)
    if a.ndim == 1:
        a = a[None, :]
    if a.ndim != 2:
        raise ValueError("x must be [n] or [batch, n]")
    return a.astype(np.float64)


def _cycles_to_unit(cyc: np.ndarray, sign: float) -> np.ndarray:
    """e^{sign * j 2 pi cyc} for phases given in cycles (already reduced)."""
    ang = 2.0 * np.pi * cyc
    return np.cos(ang) + 1j * sign * np.sin(ang)


def _dft_bins_int(xb: np.ndarray, length: int, bins: np.ndarray) -> np.ndarray:
    """X[b, j] = sum_n x[b, n] e^{-j 2 pi (bins[j] n mod length) / length}.

    Section 2.1, Eq. 2 (forward sign).  The phase index is an exact int64
    product reduced modulo ``length``; the unit-circle table is built with
    libm in float64.  One real matmul per cos / sin part.
    """
    nb, n = xb.shape
    bins = np.asarray(bins, dtype=np.int64)
    out = np.empty((nb, bins.size), dtype=np.complex128)
    tab_idx = np.arange(length, dtype=np.float64) / float(length)
    cos_t = np.cos(2.0 * np.pi * tab_idx)
    sin_t = np.sin(2.0 * np.pi * tab_idx)
    nn = np.arange(n, dtype=np.int64)
    chunk = max(1, _CHUNK_ELEMS // max(1, n))
    for c0 in range(0, bins.size, chunk):
        kk = bins[c0:c0 + chunk]
        idx = np.mod(np.outer(nn, kk), length)          # exact: int64
        out[:, c0:c0 + chunk] = xb @ cos_t[idx] - 1j * (xb @ sin_t[idx])
    return out


# --------------------------------------------------------------------------
# Zero-padded FFT (Section 2.1, Eq. 2-3 and the zero-padding paragraph)
# --------------------------------------------------------------------------

def fft_padded(x, n_fft: int) -> np.ndarray:
    """Spectrum of real traces zero-padded to ``n_fft`` samples.

    X[k] = sum_{n<N} x[n] e^{-j 2 pi k n / N_FFT},  k = 0 .. N_FFT/2
    (Section 2.1, Eq. 2 with the forward sign; padding appends zeros, so the
    sum stops at the trace length N).  Unnormalised.  Returns complex128
    [batch, N_FFT/2 + 1].
    """
    xb = _as_batch(x)
    if n_fft < xb.shape[1]:
        raise ValueError("n_fft must be >= n (the paper pads, never truncates)")
    return _dft_bins_int(xb, n_fft, np.arange(n_fft // 2 + 1))


def fft_padded_bins(x, n_fft: int, bins) -> np.ndarray:
    """``fft_padded`` restricted to the listed bin indices (0 <= k <= N_FFT/2)."""
    xb = _as_batch(x)
    return _dft_bins_int(xb, n_fft, np.asarray(bins))


# --------------------------------------------------------------------------
# Chirp-z transform on the unit circle (Section 2.3, Eq. 11, 16-23)
# --------------------------------------------------------------------------

def czt_step(f1: float, f2: float, m: int) -> float:
    """Bin spacing of the CZT grid: (f2 - f1)/(M - 1), both band edges being
    bins (Eq. 18); 0 for a single bin."""
    return 0.0 if m <= 1 else (f2 - f1) / (m - 1)


def czt_grid(fs: float, f1: float, f2: float, m: int) -> np.ndarray:
    """Frequencies f_k = f1 + k (f2 - f1)/(M - 1) of the CZT bins, k < M."""
    return f1 + np.arange(m) * czt_step(f1, f2, m)


def _czt_cycles(n: np.ndarray, k: np.ndarray, a: float, b: float) -> np.ndarray:
    """Phase of A^{-n} W^{kn} in cycles, reduced: frac(a n) + frac(b (k n)).

    A = e^{j 2 pi a} (Eq. 16 with A_0 = 1, a = f1/fs) and
    W = e^{-j 2 pi b} (Eq. 17 with W_0 = 1, b = step/fs).  k n is an exact
    int64 product before the float64 multiply.
    """
    an = np.mod(a * n.astype(np.float64), 1.0)[:, None]
    kn = np.outer(n, k).astype(np.float64)              # exact below 2^53
    bkn = np.mod(b * kn, 1.0)
    return an + bkn


def czt_bins(x, fs: float, f1: float, f2: float, m: int, bins) -> np.ndarray:
    """CZT X[k] = sum_n x[n] A^{-n} W^{kn} (Eq. 11) at the listed k < M.

    A = e^{j 2 pi f1/fs}, W = e^{-j 2 pi step/fs}, step = (f2 - f1)/(M - 1);
    i.e. the samples of the trace's z-transform at z_k = e^{j 2 pi f_k/fs}
    on the unit circle (Eq. 16-17 with A_0 = W_0 = 1).  Unnormalised.
    """
    xb = _as_batch(x)
    nb, n = xb.shape
    a = f1 / fs
    b = czt_step(f1, f2, m) / fs
    bins = np.asarray(bins, dtype=np.int64)
    out = np.empty((nb, bins.size), dtype=np.complex128)
    nn = np.arange(n, dtype=np.int64)
    chunk = max(1, _CHUNK_ELEMS // max(1, n))
    for c0 in range(0, bins.size, chunk):
        kk = bins[c0:c0 + chunk]
        cyc = _czt_cycles(nn, kk, a, b)
        ang = 2.0 * np.pi * cyc
        # z_k^{-n} = e^{-j 2 pi (a n + b k n)}
        out[:, c0:c0 + chunk] = xb @ np.cos(ang) - 1j * (xb @ np.sin(ang))
    return out


def czt(x, fs: float, f1: float, f2: float, m: int) -> np.ndarray:
    """All M bins of ``czt_bins``: complex128 [batch, M]."""
    return czt_bins(x, fs, f1, f2, m, np.arange(m))


def czt_spiral_bins(x, fs: float, f1: float, f2: float, m: int, a0: float, w0: float, bins) -> np.ndarray:
    """CZT off the unit circle (Eq. 11 with Eq. 16-17): X[k] = sum_n x[n] A^{-n} W^{kn}
    at the listed k < M, A = a0 e^{j 2 pi f1/fs}, W = w0 e^{-j 2 pi step/fs},
    i.e. the z-transform on the spiral z_k = A W^{-k}.  The magnitude of
    A^{-n} W^{kn} is exp(-n ln a0 + k n ln w0) (k n exact in int64); the phase is
    the unit-circle one.  a0 = w0 = 1 gives ``czt_bins``.
    """
    xb = _as_batch(x)
    nb, n = xb.shape
    a = f1 / fs
    b = czt_step(f1, f2, m) / fs
    la, lw = math.log(a0), math.log(w0)
    bins = np.asarray(bins, dtype=np.int64)
    out = np.empty((nb, bins.size), dtype=np.complex128)
    nn = np.arange(n, dtype=np.int64)
    chunk = max(1, _CHUNK_ELEMS // max(1, n))
    for c0 in range(0, bins.size, chunk):
        kk = bins[c0:c0 + chunk]
        ang = 2.0 * np.pi * _czt_cycles(nn, kk, a, b)
        mag = np.exp(-la * nn.astype(np.float64)[:, None] + lw * np.outer(nn, kk).astype(np.float64))
        out[:, c0:c0 + chunk] = xb @ (mag * np.cos(ang)) - 1j * (xb @ (mag * np.sin(ang)))
    return out


def czt_spiral(x, fs: float, f1: float, f2: float, m: int, a0: float, w0: float) -> np.ndarray:
    """All M bins of ``czt_spiral_bins``: complex128 [batch, M]."""
    return czt_spiral_bins(x, fs, f1, f2, m, a0, w0, np.arange(m))


# --------------------------------------------------------------------------
# Zoom FFT (Section 2.2, Eq. 6-10): mix, low-pass FIR, decimate, FFT
# --------------------------------------------------------------------------

def zoom_lout(n: int, n_taps: int, d: int) -> int:
    """Number of decimated samples u[m] kept: the full convolution's length
    N + L_h - 1 sampled every D-th point, i.e. ceil((N + L_h - 1)/D)."""
    return (n + n_taps - 1 + d - 1) // d


def zoom_grid(fs: float, f1: float, f2: float, d: int, n_fft: int) -> np.ndarray:
    """Frequencies of the K = N_FFT/D zoom bins: f_N + (i - K/2) fs/N_FFT."""
    k = n_fft // d
    fn = 0.5 * (f1 + f2)
    return fn + (np.arange(k) - k // 2) * (fs / n_fft)


def _zoom_decimated(xb: np.ndarray, fs: float, f1: float, f2: float, d: int,
                    taps: np.ndarray) -> np.ndarray:
    """Steps 1-3 of the Zoom FFT for each trace: u[m] = (h * y)[m D]."""
    nb, n = xb.shape
    h = np.asarray(taps, dtype=np.float64)
    # Eq. 6: band centre.
    fn = 0.5 * (f1 + f2)
    # Eq. 7 (read as a down-shift by f_N): y[n] = x[n] e^{-j 2 pi f_N n / fs},
    # phase in cycles reduced to [0, 1) before the trig call.
    cyc = np.mod((fn / fs) * np.arange(n, dtype=np.float64), 1.0)
    mix = _cycles_to_unit(cyc, -1.0)
    lout = zoom_lout(n, h.size, d)
    u = np.empty((nb, lout), dtype=np.complex128)
    for b in range(nb):
        y = xb[b] * mix
        # Eq. 8/10: causal FIR, zero initial state, full linear convolution.
        z = np.convolve(h, y)                            # length N + L_h - 1
        # Eq. 9-10: keep every D-th output, starting at m = 0.
        u[b] = z[::d][:lout]
    return u


def zoom_bins(x, fs: float, f1: float, f2: float, d: int, taps, n_fft: int,
              bins) -> np.ndarray:
    """Zoom-FFT output bins ``bins`` (0 <= i < K) in ascending frequency.

    out[i] = U[(i - K/2) mod K], U[j] = sum_m u[m] e^{-j 2 pi j m / K},
    K = N_FFT / D; u from ``_zoom_decimated``.
    """
    xb = _as_batch(x)
    if n_fft % d != 0:
        raise ValueError("n_fft must be a multiple of d")
    k = n_fft // d
    u = _zoom_decimated(xb, fs, f1, f2, d, np.asarray(taps))
    if u.shape[1] > k:
        raise ValueError("ceil((N + L_h - 1)/D) must not exceed N_FFT/D")
    bins = np.asarray(bins, dtype=np.int64)
    j = np.mod(bins - k // 2, k)                         # fftshift
    # K-point DFT of the L_out kept samples (the rest of the K are zeros).
    nn = np.arange(u.shape[1], dtype=np.int64)
    tab = np.arange(k, dtype=np.float64) / float(k)
    cos_t = np.cos(2.0 * np.pi * tab)
    sin_t = np.sin(2.0 * np.pi * tab)
    out = np.empty((xb.shape[0], bins.size), dtype=np.complex128)
    chunk = max(1, _CHUNK_ELEMS // max(1, nn.size))
    for c0 in range(0, j.size, chunk):
        idx = np.mod(np.outer(nn, j[c0:c0 + chunk]), k)
        e = cos_t[idx] - 1j * sin_t[idx]
        out[:, c0:c0 + chunk] = u @ e
    return out


def zoom(x, fs: float, f1: float, f2: float, d: int, taps, n_fft: int) -> np.ndarray:
    """All K = N_FFT/D zoom bins: complex128 [batch, K]."""
    return zoom_bins(x, fs, f1, f2, d, taps, n_fft, np.arange(n_fft // d))


# --------------------------------------------------------------------------
# Helpers that follow the paper's resolution formulas
# --------------------------------------------------------------------------

def fft_resolution(fs: float, n_fft: int) -> float:
    """Delta f = fs / N_FFT (Section 2.1, Eq. 3)."""
    return fs / n_fft


def czt_resolution_eq24(f1: float, f2: float, m: int) -> float:
    """The paper's CZT resolution (f_max - f_min)/N_CZT (Section 2.3, Eq. 24)."""
    return (f2 - f1) / m


def zeros_for_delta(fs: float, n_fft: int, delta: float) -> int:
    """Zeros x to append so that the resolution improves by ``delta``.

    Section 2.1, Eq. 4-5: Delta = fs/N_FFT - fs/(N_FFT + x), solved for x:
    x = fs N_FFT / (fs - Delta N_FFT) - N_FFT ("L" in Eq. 5 is N_FFT).
    The smallest integer x whose improvement reaches ``delta`` is returned.
    """
    if not (fs > 0 and n_fft > 0 and delta >= 0 and delta * n_fft < fs):
        raise ValueError("need fs > 0, n_fft > 0 and 0 <= delta < fs/n_fft")
    xr = fs * n_fft / (fs - delta * n_fft) - n_fft
    x = max(0, math.ceil(xr - 1e-9 * max(1.0, abs(xr))))
    while fs / n_fft - fs / (n_fft + x) < delta * (1.0 - 1e-12):
        x += 1
    return x


def m_for_resolution(fs: float, f1: float, f2: float, n_fft: int) -> int:
    """CZT points for the FFT's resolution: N_CZT = (f2 - f1)/fs * N_FFT
    (Section 2.3, Eq. 25), rounded up to an integer."""
    v = abs(f2 - f1) / fs * n_fft
    return max(1, math.ceil(v - 1e-9 * max(1.0, v)))


def design_lowpass(n_taps: int, d: int) -> np.ndarray:
    """Low-pass FIR for the Zoom FFT decimator (Section 2.2, Eq. 8 realised
    as a finite filter).

    Hamming-windowed sinc with cutoff f_c = fs/(2D):
    h[k] = w[k] (1/D) sinc((k - (L_h - 1)/2)/D),
    w[k] = 0.54 - 0.46 cos(2 pi k/(L_h - 1)), then scaled so that sum h = D
    (the gain C of Eq. 8 is taken as D, so in-band bins keep the scale of
    the undecimated spectrum).
    """
    if n_taps < 1 or d < 1:
        raise ValueError("n_taps >= 1 and d >= 1")
    k = np.arange(n_taps, dtype=np.float64)
    if n_taps == 1:
        w = np.ones(1)
    else:
        w = 0.54 - 0.46 * np.cos(2.0 * np.pi * k / (n_taps - 1))
    h = w * np.sinc((k - 0.5 * (n_taps - 1)) / d) / d
    return h * (d / h.sum())
