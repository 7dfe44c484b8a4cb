"""Seeded synthetic THz-TDS traces.

The paper's experimental traces (Section 3.2: T_s = 100 fs, N = 500 samples)
are not published with it, so the workloads use a stand-in with their shape:
a single-cycle pulse (first derivative of a Gaussian), delayed scaled echoes,
and white Gaussian noise at a stated peak-amplitude SNR.  This module holds no
transform arithmetic; it only draws inputs.  The same float32 arrays feed the
CUDA library and the FP64 oracle.

Every trace draws from its own ``numpy.random.Generator`` seeded with
``[workload_id, trace_index]``, so any trace can be regenerated alone.

Workloads (ids 0-4):
  0  one trace, N = 2048, fs = 20 THz, sigma 0.25 ps at 15 ps, echo +6 ps x0.3,
     60 dB; FFT to 16384, CZT 0.2-2.5 THz at M = 1024, Zoom centred 1.35 THz,
     D = 4, 63 taps.
  1  4096 traces like 0 with per-trace jitter (sigma 0.2-0.35 ps, delay
     10-20 ps, echo 2-10 ps at 0.1-0.5, SNR 40-70 dB), same transform sizes.
  2  10000 ragged traces, N in [1000, 8192]; per-trace band f1 in
     [0.1, 1.0] THz, width [0.5, 3.0] THz, M in [256, 4096]; D in {2,4,8,16};
     odd tap count in [31, 127]; N_FFT = 8 * nextpow2(N).
  3  65536 traces, N = 1024, band 0.8-1.2 THz at M = 512.
  4  256 traces, N = 262144, pulse at 15 ps plus 8 echoes at 0.1-13 ns with
     amplitude 0.5^j, 60 dB; FFT to 2^21, CZT 0.3-0.4 THz at M = 65536, Zoom
     centred 0.35 THz with D = 64 and 255 taps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

THZ = 1e12
PS = 1e-12
NS = 1e-9
FS = 20 * THZ


def pulse(t: np.ndarray, t0: float, sigma: float) -> np.ndarray:
    """Gaussian-derivative pulse -(t - t0)/sigma^2 exp(-(t - t0)^2/(2 sigma^2)),
    scaled to a peak of 1 (the peak sits at t0 - sigma)."""
    u = t - t0
    return -u / sigma * np.exp(0.5 - 0.5 * (u / sigma) ** 2)


def trace(n: int, fs: float, sigma: float, t0: float, echoes, snr_db: float,
          rng: np.random.Generator | None) -> np.ndarray:
    """One float32 trace: pulse(t0) + sum_j a_j pulse(t0 + tau_j) + noise.

    ``echoes`` is a sequence of (delay tau_j, amplitude a_j).  Noise is white
    Gaussian with sigma_noise = max|s| 10^{-SNR/20}; ``rng=None`` gives the
    noise-free trace.
    """
    t = np.arange(n, dtype=np.float64) / fs
    s = pulse(t, t0, sigma)
    for tau, amp in echoes:
        s = s + amp * pulse(t, t0 + tau, sigma)
    if rng is not None:
        s = s + rng.normal(0.0, np.max(np.abs(s)) * 10.0 ** (-snr_db / 20.0), n)
    return s.astype(np.float32)


def trace_rng(workload: int, index: int) -> np.random.Generator:
    return np.random.default_rng([int(workload), int(index)])


def nextpow2(v: int) -> int:
    return 1 if v <= 1 else 1 << (int(v) - 1).bit_length()


@dataclass
class Uniform:
    """Transform parameters shared by every trace of a batch."""
    workload: int
    batch: int
    n: int
    fs: float
    n_fft: int
    czt_f1: float
    czt_f2: float
    czt_m: int
    zoom_f1: float
    zoom_f2: float
    zoom_d: int
    zoom_taps: int
    zoom_n_fft: int


UNIFORM = {
    0: Uniform(0, 1, 2048, FS, 16384, 0.2 * THZ, 2.5 * THZ, 1024,
               0.2 * THZ, 2.5 * THZ, 4, 63, 16384),
    1: Uniform(1, 4096, 2048, FS, 16384, 0.2 * THZ, 2.5 * THZ, 1024,
               0.2 * THZ, 2.5 * THZ, 4, 63, 16384),
    3: Uniform(3, 65536, 1024, FS, 8192, 0.8 * THZ, 1.2 * THZ, 512,
               0.8 * THZ, 1.2 * THZ, 4, 63, 8192),
    4: Uniform(4, 256, 262144, FS, 1 << 21, 0.3 * THZ, 0.4 * THZ, 65536,
               0.3 * THZ, 0.4 * THZ, 64, 255, 1 << 21),
}


def _trace_for(workload: int, i: int, n: int) -> np.ndarray:
    rng = trace_rng(workload, i)
    if workload == 0:
        return trace(n, FS, 0.25 * PS, 15 * PS, [(6 * PS, 0.3)], 60.0, rng)
    if workload == 4:
        delays = np.sort(rng.uniform(0.1 * NS, 13 * NS, 8))
        echoes = [(float(dl) - 15 * PS, 0.5 ** (j + 1)) for j, dl in enumerate(delays)]
        return trace(n, FS, 0.25 * PS, 15 * PS, echoes, 60.0, rng)
    sigma = rng.uniform(0.2, 0.35) * PS
    t0 = rng.uniform(10, 20) * PS
    tau = rng.uniform(2, 10) * PS
    amp = rng.uniform(0.1, 0.5)
    snr = rng.uniform(40, 70)
    return trace(n, FS, sigma, t0, [(tau, amp)], snr, rng)


def batch_traces(workload: int, indices, n: int | None = None) -> np.ndarray:
    """float32 [len(indices), N] traces of a uniform workload (0, 1, 3, 4)."""
    cfg = UNIFORM[workload]
    n = cfg.n if n is None else n
    idx = list(indices)
    out = np.empty((len(idx), n), dtype=np.float32)
    for r, i in enumerate(idx):
        out[r] = _trace_for(workload, i, n)
    return out


@dataclass
class RaggedTrace:
    n: int
    n_fft: int
    f1: float
    f2: float
    m: int
    d: int
    n_taps: int


@dataclass
class Ragged:
    """Workload 2: per-trace length, band, point count, decimation and taps."""
    items: list = field(default_factory=list)
    fs: float = FS


def ragged_params(count: int = 10000, workload: int = 2) -> Ragged:
    rg = Ragged()
    for i in range(count):
        rng = trace_rng(workload, i)
        n = int(rng.integers(1000, 8193))
        f1 = rng.uniform(0.1, 1.0) * THZ
        width = rng.uniform(0.5, 3.0) * THZ
        m = int(rng.integers(256, 4097))
        d = int(rng.choice([2, 4, 8, 16]))
        taps = int(rng.integers(15, 64)) * 2 + 1          # odd, 31 .. 127
        rg.items.append(RaggedTrace(n, 8 * nextpow2(n), f1, f1 + width, m, d, taps))
    return rg


def ragged_trace(i: int, item: RaggedTrace, workload: int = 2) -> np.ndarray:
    """Trace i of the ragged workload (jitter as in workload 1)."""
    rng = trace_rng(workload * 1000 + 1, i)
    sigma = rng.uniform(0.2, 0.35) * PS
    t0 = rng.uniform(10, 20) * PS
    tau = rng.uniform(2, 10) * PS
    amp = rng.uniform(0.1, 0.5)
    snr = rng.uniform(40, 70)
    return trace(item.n, FS, sigma, t0, [(tau, amp)], snr, rng)
