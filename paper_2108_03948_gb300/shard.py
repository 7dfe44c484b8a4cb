"""Partition a batch of traces across the ranks of a multi-GPU job.

Every spectrum of the method is a sum over one trace's own samples (the DFT of
Section 2.1, Eq. 2; the chirp-z of Section 2.3, Eq. 11; the Zoom FFT of
Section 2.2, Eq. 6-10), so traces are independent and a batch shards by trace
with no exchange between GPUs.  This module is pure host logic: it decides
which rank transforms which traces and how the per-rank spectra go back into
the single-rank order.  No collective is on the data path; the benchmark only
reduces its elapsed time (a max over ranks).

* ``contiguous_slices`` -- a uniform batch (every trace costs the same):
  contiguous runs whose lengths differ by at most one trace.
* ``balance_by_cost`` -- a ragged batch: the greedy longest-processing-time
  rule (traces by decreasing estimated cost, each to the rank with the least
  load so far); each rank's list is returned in ascending trace order.
* ``ragged_trace_cost`` -- the estimate it balances: the three transforms'
  modelled GPU time of one trace (algorithmic bytes at the HBM rate plus
  algorithmic flops at the FP32 rate, whichever is longer, per transform).
* ``assemble`` -- put per-rank results back in the order of the whole batch.
"""
from __future__ import annotations

import heapq
import math
from typing import Iterable, Sequence

# Modelled rates of one GB300 (the cost model only needs their ratio).
HBM_BYTES_PER_S = 6.78e12
FP32_FLOP_PER_S = 7.4e13


def contiguous_slices(total: int, world: int) -> list[tuple[int, int]]:
    """Split ``range(total)`` into ``world`` contiguous [start, stop) runs;
    the first ``total % world`` runs hold one trace more."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if total < 0:
        raise ValueError("total must be >= 0")
    base, extra = divmod(total, world)
    out, start = [], 0
    for r in range(world):
        stop = start + base + (1 if r < extra else 0)
        out.append((start, stop))
        start = stop
    return out


def _bluestein_length(n: int, m: int) -> int:
    return max(16, 1 << (n + m - 2).bit_length())


def ragged_trace_cost(n: int, n_fft: int, m: int, d: int, n_taps: int) -> float:
    """Modelled seconds of one ragged trace through the three transforms:
    per transform max(bytes / HBM rate, flops / FP32 rate), with bytes the
    input read once and the output written once, and flops the usual counts
    (5 L log2 L per complex L-point FFT, half for real input; Bluestein two
    L-point FFTs plus the chirp products; Zoom the FIR at the kept outputs
    plus its K-point FFT)."""
    def t(nbytes, flops):
        return max(nbytes / HBM_BYTES_PER_S, flops / FP32_FLOP_PER_S)
    fft = t(4 * n + 8 * (n_fft // 2 + 1), 2.5 * n_fft * math.log2(max(n_fft, 2)))
    L = _bluestein_length(n, m)
    czt = t(4 * n + 8 * m, 10 * L * math.log2(L) + 6 * (n + L + m))
    K = max(1, n_fft // d)
    lout = (n + n_taps - 1 + d - 1) // d
    zoom = t(4 * n + 8 * K, 4 * lout * n_taps + 6 * n + 5 * K * math.log2(max(K, 2)))
    return fft + czt + zoom


def balance_by_cost(costs: Sequence[float], world: int) -> list[list[int]]:
    """Greedy longest-processing-time partition of trace indices into
    ``world`` lists of near-equal total cost.  Ties go to the lower rank, so
    the result is deterministic; each list is sorted ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    for p in parts:
        p.sort()
    return parts


def imbalance(costs: Sequence[float], parts: Iterable[Sequence[int]]) -> float:
    """(largest rank load - mean load) / mean load."""
    loads = [sum(float(costs[i]) for i in p) for p in parts]
    mean = sum(loads) / len(loads) if loads else 0.0
    return 0.0 if mean == 0.0 else (max(loads) - mean) / mean


def assemble(parts: Sequence[Sequence[int]], results: Sequence[Sequence], total: int) -> list:
    """Inverse of a partition: ``results[r][j]`` belongs to trace
    ``parts[r][j]``; returns the list of all ``total`` results in trace order.
    Raises if a trace is missing or assigned twice."""
    out: list = [None] * total
    seen = [False] * total
    for p, res in zip(parts, results):
        if len(p) != len(res):
            raise ValueError("a rank returned a different number of results than traces")
        for i, v in zip(p, res):
            if seen[i]:
                raise ValueError(f"trace {i} assigned twice")
            seen[i] = True
            out[i] = v
    if not all(seen):
        raise ValueError(f"trace {seen.index(False)} assigned to no rank")
    return out


def slices_as_parts(slices: Sequence[tuple[int, int]]) -> list[list[int]]:
    return [list(range(a, b)) for a, b in slices]
