"""Section 3.1's two-tone experiment through the CUDA path: the spectra of
the GPU FFT (N_FFT = 1138, a chirp-z on the DFT grid) and chirp-z (7.03 Hz
grid) match the FP64 oracle, and both first resolve the tones at the same
separation as the oracle does."""
import numpy as np
import pytest

from oracle import spec_oracle as O
from paper_2108_03948_gb300.two_tone import dip_ratio

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FS, N, F1, F2, M, FA = 8000.0, 128, 100.0, 1000.0, 128, 400.0
F2P = F1 + (F2 - F1) * (M - 1) / M
NFFT = 1138


def test_two_tone_spectra_and_resolution():
    from paper_2108_03948_gb300 import build
    build.build()
    from paper_2108_03948_gb300 import spec
    deltas = np.arange(20.0, 141.0, 5.0)
    t = np.arange(N) / FS
    x = np.stack([np.sin(2 * np.pi * FA * t) + np.sin(2 * np.pi * (FA + d) * t) for d in deltas]).astype(np.float32)
    with spec.Context(0) as ctx:
        xd = torch.from_numpy(x).cuda()
        X = spec.spec_fft(ctx, xd, FS, NFFT).cpu().numpy()
        Z = spec.spec_czt(ctx, xd, FS, F1, F2P, M).cpu().numpy()
    Xo = O.fft_padded(x, NFFT)
    Zo = O.czt(x, FS, F1, F2P, M)
    rel = lambda a, b: (np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)).max()
    assert rel(X, Xo) <= 1e-5 and rel(Z, Zo) <= 1e-5
    ff = np.arange(NFFT // 2 + 1) * FS / NFFT
    cf = F1 + np.arange(M) * (F2P - F1) / (M - 1)

    def first(freqs, S):
        for i, d in enumerate(deltas):
            if dip_ratio(freqs, np.abs(S[i]), FA, FA + d) < 2 ** -0.5:
                return d
    assert first(ff, X) == first(ff, Xo) == first(cf, Z) == first(cf, Zo)
