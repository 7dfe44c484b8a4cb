"""Sizes of the resolution sweep (Section 4, Fig. 11) against the paper's
formulas: N_FFT = ceil(fs / Delta f) (Eq. 3), M = ceil((f2 - f1) N_FFT / fs)
(Eq. 25, the oracle's helper), and a Zoom FFT whose K = N_FFT / D covers the
requested resolution and the decimated samples.  CPU only."""
import math

import pytest

from oracle import spec_oracle as O


@pytest.fixture(scope="module")
def sweep():
    from paper_2108_03948_gb300 import build as b
    try:
        b.build()
    except RuntimeError as e:          # no nvcc on this machine
        pytest.skip(f"cannot build the CUDA library here: {e}")
    from paper_2108_03948_gb300 import sweep as s
    return s


FS, N, F1, F2 = 10e12, 500, 0.1e12, 3.0e12


def test_zoom_decimation_keeps_the_band(sweep):
    d = sweep.zoom_decimation(FS, F1, F2)
    assert d & (d - 1) == 0
    assert FS / d >= 1.25 * (F2 - F1) > FS / (2 * d)
    assert d == 2


@pytest.mark.parametrize("i", range(40))
def test_sizes_follow_eq3_and_eq25(sweep, i):
    df = 20e9 - 0.5e9 * i
    d = sweep.zoom_decimation(FS, F1, F2)
    n_fft, m, k = sweep.sizes(FS, N, F1, F2, df, d)
    assert n_fft == max(N, math.ceil(FS / df))
    assert FS / n_fft <= df * (1 + 1e-12)                 # the FFT reaches the requested resolution
    assert m == O.m_for_resolution(FS, F1, F2, n_fft)
    assert k & (k - 1) == 0 and k * d >= n_fft             # the Zoom FFT's spacing fs/(K D) <= Delta f
    assert (N + 63 - 1 + d - 1) // d <= k                 # every decimated sample fits
    assert k // 2 * d < n_fft or (N + 63 - 1 + d - 1) // d > k // 2   # K is the smallest such power of two


def test_paper_points(sweep):
    d = sweep.zoom_decimation(FS, F1, F2)
    assert sweep.sizes(FS, N, F1, F2, 20e9, d)[0] == 500    # the unpadded 500-sample trace at 20 GHz
    assert sweep.sizes(FS, N, F1, F2, 0.5e9, d)[0] == 20000
