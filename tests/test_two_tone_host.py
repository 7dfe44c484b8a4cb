"""Section 3.1's two-tone experiment on the FP64 oracle (CPU): the dip
measure of paper_2108_03948_gb300.two_tone separates clearly resolved from
unresolved tone pairs, and -- the paper's finding -- the chirp-z at a
plotting resolution of 7.03 Hz does not resolve two tones earlier than the
zero-padded FFT at the same plotting resolution: both are bounded by the
128-sample window."""
import numpy as np

from oracle import spec_oracle as O
from paper_2108_03948_gb300.two_tone import dip_ratio

FS, N = 8000.0, 128
F1, F2, M = 100.0, 1000.0, 128
F2P = F1 + (F2 - F1) * (M - 1) / M
NFFT = int(round(FS / ((F2 - F1) / M)))
FA = 400.0


def spectra(delta):
    t = np.arange(N) / FS
    x = np.sin(2 * np.pi * FA * t) + np.sin(2 * np.pi * (FA + delta) * t)
    X = np.abs(O.fft_padded(x, NFFT)[0])
    Z = np.abs(O.czt(x, FS, F1, F2P, M)[0])
    return (np.arange(NFFT // 2 + 1) * FS / NFFT, X), (F1 + np.arange(M) * (F2P - F1) / (M - 1), Z)


def first_resolved(which):
    for d in np.arange(20.0, 201.0, 5.0):
        (ff, X), (cf, Z) = spectra(d)
        r = dip_ratio(ff, X, FA, FA + d) if which == "fft" else dip_ratio(cf, Z, FA, FA + d)
        if r < 2 ** -0.5:
            return d
    return None


def test_grids_match_the_paper():
    assert NFFT == 1138
    assert abs((F2P - F1) / (M - 1) - 7.03125) < 1e-9         # the printed 7.03 Hz


def test_dip_measure():
    (ff, X), (cf, Z) = spectra(150.0)                        # well apart: deep dip
    assert dip_ratio(ff, X, FA, FA + 150) < 0.3
    assert dip_ratio(cf, Z, FA, FA + 150) < 0.3
    (ff, X), (cf, Z) = spectra(20.0)                         # far below fs/N: one lobe
    assert dip_ratio(ff, X, FA, FA + 20) > 0.9
    assert dip_ratio(cf, Z, FA, FA + 20) > 0.9


def test_czt_does_not_resolve_earlier_than_fft():
    df, dc = first_resolved("fft"), first_resolved("czt")
    assert df is not None and dc is not None
    assert dc >= df - 5.0                                     # within one step of the sweep
    assert 40.0 <= df <= 80.0                                 # of the order of fs/N = 62.5 Hz
