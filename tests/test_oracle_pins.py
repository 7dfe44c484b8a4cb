"""Pins for the FP64 oracle: each test checks it against something other than
itself -- a library routine computing the same quantity by another algorithm,
a closed form, an invariant, or a number printed in the paper.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
import scipy.signal as sps

from oracle import spec_oracle as O
from paper_2108_03948_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.json")


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def rnd(n, seed, batch=None):
    g = np.random.default_rng(seed)
    shape = (n,) if batch is None else (batch, n)
    return g.standard_normal(shape)


# ---------------------------------------------------------------- FFT ------

@pytest.mark.parametrize("n,n_fft", [(1, 1), (1, 8), (5, 8), (37, 64), (300, 512),
                                     (300, 300), (129, 1000), (2048, 16384)])
def test_fft_matches_library_rfft(n, n_fft):
    # numpy's pocketfft: a different algorithm for the same padded DFT (Eq. 2).
    x = rnd(n, 1, batch=3)
    got = O.fft_padded(x, n_fft)
    ref = np.fft.rfft(x, n_fft, axis=1)
    assert got.shape == (3, n_fft // 2 + 1)
    assert rel(got, ref) < 1e-12


def test_fft_tone_on_bin_is_a_delta():
    n = 256
    k0 = 37
    x = np.cos(2 * np.pi * k0 * np.arange(n) / n)
    X = O.fft_padded(x, n)[0]
    expect = np.zeros(n // 2 + 1, complex)
    expect[k0] = n / 2
    assert np.max(np.abs(X - expect)) < 1e-10


def test_fft_zero_padding_interpolates_unpadded_bins():
    # Section 2.1: padding adds no information; bin k*P of the padded FFT is
    # bin k of the unpadded DFT (checked against the library's unpadded FFT).
    n, p = 200, 8
    x = rnd(n, 2)
    Xp = O.fft_padded(x, n * p)[0]
    ref = np.fft.fft(x)[: n // 2 + 1]
    assert rel(Xp[::p], ref) < 1e-12


def test_fft_parseval():
    n, n_fft = 700, 4096
    x = rnd(n, 3)
    X = O.fft_padded(x, n_fft)[0]
    e_freq = (abs(X[0]) ** 2 + 2 * np.sum(abs(X[1:-1]) ** 2) + abs(X[-1]) ** 2) / n_fft
    assert abs(e_freq - np.sum(x ** 2)) / np.sum(x ** 2) < 1e-12


def test_fft_impulse_closed_form():
    n, n_fft, n0 = 64, 512, 17
    x = np.zeros(n)
    x[n0] = 1.0
    k = np.arange(n_fft // 2 + 1)
    expect = np.exp(-2j * np.pi * k * n0 / n_fft)
    assert np.max(np.abs(O.fft_padded(x, n_fft)[0] - expect)) < 1e-13


def dirichlet(n, w):
    """sum_{n<N} e^{-j w n} in closed form."""
    w = np.asarray(w, float)
    out = np.empty(w.shape, complex)
    small = np.abs(np.sin(w / 2)) < 1e-300
    ws = w[~small]
    out[~small] = np.exp(-0.5j * ws * (n - 1)) * np.sin(n * ws / 2) / np.sin(ws / 2)
    out[small] = n * np.exp(-0.5j * w[small] * (n - 1))
    return out


def test_fft_constant_is_dirichlet_kernel():
    n, n_fft = 100, 1024
    k = np.arange(n_fft // 2 + 1)
    expect = dirichlet(n, 2 * np.pi * k / n_fft)
    assert np.max(np.abs(O.fft_padded(np.ones(n), n_fft)[0] - expect)) < 1e-10


def pulse_spectrum(f, fs, t0, sigma, echoes):
    """Sampled-trace DTFT fs * P(f) of the peak-normalised Gaussian-derivative
    pulse plus echoes: P(f) = sigma e^{1/2} j 2 pi f sigma sqrt(2 pi)
    e^{-2 pi^2 sigma^2 f^2} e^{-j 2 pi f t0} (1 + sum a e^{-j 2 pi f tau})."""
    g = sigma * np.exp(0.5) * 2j * np.pi * f * sigma * np.sqrt(2 * np.pi) \
        * np.exp(-2 * np.pi ** 2 * sigma ** 2 * f ** 2) * np.exp(-2j * np.pi * f * t0)
    e = 1.0 + sum(a * np.exp(-2j * np.pi * f * tau) for tau, a in echoes)
    return fs * g * e


def test_fft_pulse_closed_form():
    # Noise-free workload-0 pulse: aliasing (e^-123) and truncation (e^-1800)
    # are far below float64, so the DFT equals fs * P(f_k) at f_k = k fs/N_FFT.
    fs, n, n_fft = synth.FS, 2048, 16384
    sigma, t0, echoes = 0.25 * synth.PS, 15 * synth.PS, [(6 * synth.PS, 0.3)]
    x = synth.pulse(np.arange(n) / fs, t0, sigma) \
        + 0.3 * synth.pulse(np.arange(n) / fs, t0 + 6 * synth.PS, sigma)
    X = O.fft_padded(x, n_fft)[0]
    f = np.arange(n_fft // 2 + 1) * fs / n_fft
    ref = pulse_spectrum(f, fs, t0, sigma, echoes)
    assert rel(X, ref) < 1e-11


# ---------------------------------------------------------------- CZT ------

def test_czt_reduces_to_dft():
    # Section 2.3 after Eq. 11: A = 1, W = e^{-j2pi/N}, N_CZT = N gives the DFT.
    n = 96
    fs = 1000.0
    x = rnd(n, 4)
    X = O.czt(x, fs, 0.0, fs * (n - 1) / n, n)[0]
    assert rel(X, np.fft.fft(x)) < 1e-12


@pytest.mark.parametrize("n,m,f1,f2", [(128, 128, 100.0, 1000.0), (333, 77, 1234.0, 987.0),
                                       (50, 400, -300.0, 3900.0), (64, 1, 250.0, 250.0)])
def test_czt_matches_library_czt(n, m, f1, f2):
    # scipy's chirp-z (Bluestein, a different algorithm) on z_k = a w^{-k}.
    fs = 8000.0
    x = rnd(n, 5, batch=2)
    step = O.czt_step(f1, f2, m)
    a = np.exp(2j * np.pi * f1 / fs)
    w = np.exp(-2j * np.pi * step / fs)
    ref = sps.czt(x, m, w, a, axis=-1)
    got = O.czt(x, fs, f1, f2, m)
    assert rel(got, ref) < 1e-9


@pytest.mark.parametrize("n,m,f1,f2,a0,w0", [(100, 64, 100.0, 1000.0, 0.98, 1.002),
                                               (160, 97, 2500.0, 300.0, 1.05, 0.999),
                                               (77, 1, 250.0, 250.0, 1.1, 0.9995)])
def test_czt_spiral_matches_library_czt(n, m, f1, f2, a0, w0):
    # off the unit circle (Eq. 16-17 with A_0, W_0 != 1): scipy's chirp-z on
    # z_k = a w^{-k} with the complex a = A, w = W
    fs = 8000.0
    x = rnd(n, 11, batch=2)
    step = O.czt_step(f1, f2, m)
    a = a0 * np.exp(2j * np.pi * f1 / fs)
    w = w0 * np.exp(-2j * np.pi * step / fs)
    ref = sps.czt(x, m, w, a, axis=-1)
    assert rel(O.czt_spiral(x, fs, f1, f2, m, a0, w0), ref) < 1e-9


def test_czt_spiral_geometric_closed_form():
    # x[n] = r^n: X[k] = sum_n (r A^{-1} W^k)^n = (1 - q^N)/(1 - q), q = r W^k / A
    n, m, fs, f1, f2, a0, w0, r = 300, 50, 10e12, 0.3e12, 2.2e12, 0.995, 1.0004, 0.99
    x = r ** np.arange(n)
    step = O.czt_step(f1, f2, m)
    A = a0 * np.exp(2j * np.pi * f1 / fs)
    W = w0 * np.exp(-2j * np.pi * step / fs)
    q = r * W ** np.arange(m) / A
    ref = (1 - q ** n) / (1 - q)
    assert rel(O.czt_spiral(x, fs, f1, f2, m, a0, w0)[0], ref) < 1e-11


def test_czt_spiral_on_the_unit_circle_is_the_czt():
    x = rnd(500, 12, batch=2)
    assert rel(O.czt_spiral(x, 10e12, 0.3e12, 2.9e12, 333, 1.0, 1.0), O.czt(x, 10e12, 0.3e12, 2.9e12, 333)) < 1e-14


def test_czt_on_fft_grid_equals_padded_fft_bins():
    n, n_fft, k1, m = 300, 2048, 123, 257
    fs = 20e12
    x = rnd(n, 6)
    got = O.czt(x, fs, k1 * fs / n_fft, (k1 + m - 1) * fs / n_fft, m)[0]
    ref = np.fft.rfft(x, n_fft)[k1:k1 + m]
    assert rel(got, ref) < 1e-11


def test_czt_constant_dirichlet_off_grid():
    n, m, fs, f1, f2 = 500, 301, 10e12, 0.137e12, 2.71e12
    got = O.czt(np.ones(n), fs, f1, f2, m)[0]
    f = O.czt_grid(fs, f1, f2, m)
    assert np.max(np.abs(got - dirichlet(n, 2 * np.pi * f / fs))) < 1e-9


def test_czt_pulse_closed_form_off_grid():
    fs, n = synth.FS, 2048
    sigma, t0 = 0.25 * synth.PS, 15 * synth.PS
    x = synth.pulse(np.arange(n) / fs, t0, sigma)
    f1, f2, m = 0.2e12, 2.5e12, 1024
    got = O.czt(x, fs, f1, f2, m)[0]
    ref = pulse_spectrum(O.czt_grid(fs, f1, f2, m), fs, t0, sigma, [])
    assert rel(got, ref) < 1e-11


def test_czt_long_phase_reduction():
    # Workload-4 scale phases (k n up to 1.7e10): a sparse trace's bin against
    # the direct sum with phases reduced exactly (Fractions of the same
    # float64 a = f1/fs and b = step/fs).
    from fractions import Fraction
    fs, f1, f2, m, n = 20e12, 0.3e12, 0.4e12, 65536, 262144
    k = 65000
    nn = np.arange(5, n, 4099)
    x = np.zeros(n)
    x[nn] = np.random.default_rng(7).standard_normal(nn.size)
    got = O.czt_bins(x, fs, f1, f2, m, [k])[0, 0]
    a = Fraction(f1 / fs)
    b = Fraction(O.czt_step(f1, f2, m) / fs)
    ph = np.array([float((a * int(v) + b * (k * int(v))) % 1) for v in nn])
    ref = np.sum(x[nn] * np.exp(-2j * np.pi * ph))
    assert abs(got - ref) / np.sum(np.abs(x[nn])) < 1e-10


# --------------------------------------------------------------- Zoom ------

def test_zoom_without_filter_or_decimation_is_shifted_czt():
    # D = 1, h = [1]: mix + K-point DFT is the CZT on the grid
    # f_N + (i - K/2) fs/N_FFT (library czt as the reference).
    n, n_fft, fs = 200, 512, 20e12
    f1, f2 = 1.0e12, 3.0e12
    x = rnd(n, 8)
    got = O.zoom(x, fs, f1, f2, 1, np.ones(1), n_fft)[0]
    grid = O.zoom_grid(fs, f1, f2, 1, n_fft)
    ref = sps.czt(x, n_fft, np.exp(-2j * np.pi * fs / n_fft / fs), np.exp(2j * np.pi * grid[0] / fs))
    assert rel(got, ref) < 1e-10


@pytest.mark.parametrize("n,d,taps,n_fft", [(256, 4, 31, 2048), (301, 3, 10, 1206), (512, 8, 63, 4096)])
def test_zoom_alias_identity(n, d, taps, n_fft):
    # The DTFT of u[m] = (h * y)[mD] is (1/D) sum_r H(nu_r) X(nu_r + 2 pi f_N/fs),
    # nu_r = (omega - 2 pi r)/D, because the full convolution is kept.  H and X
    # are evaluated here by their own direct sums at those frequencies.
    fs, f1, f2 = 20e12, 0.9e12, 1.7e12
    x = rnd(n, 9)
    h = np.random.default_rng(10).standard_normal(taps)
    got = O.zoom(x, fs, f1, f2, d, h, n_fft)[0]
    k = n_fft // d
    omega = 2 * np.pi * (np.arange(k) - k // 2) / k
    c = 0.5 * (f1 + f2) / fs
    ref = np.zeros(k, complex)
    for r in range(d):
        nu = (omega - 2 * np.pi * r) / d
        H = np.exp(-1j * np.outer(nu, np.arange(taps))) @ h
        X = np.exp(-1j * np.outer(nu + 2 * np.pi * c, np.arange(n))) @ x
        ref += H * X
    ref /= d
    assert rel(got, ref) < 1e-9


def test_zoom_tone_lands_on_its_bin():
    fs, n, n_fft, d = 20e12, 2048, 8192, 4
    f1, f2 = 1.0e12, 1.7e12
    fn = 0.5 * (f1 + f2)
    i0 = 37
    f = fn + i0 * fs / n_fft
    x = np.cos(2 * np.pi * f * np.arange(n) / fs)
    h = O.design_lowpass(63, d)
    out = O.zoom(x, fs, f1, f2, d, h, n_fft)[0]
    assert int(np.argmax(np.abs(out))) == n_fft // d // 2 + i0


def test_zoom_in_band_approximates_czt():
    # With the Hamming low-pass (gain D) the in-band zoom bins follow the
    # spectrum on the same grid up to passband ripple / stop-band leakage.
    fs, n, n_fft, d = synth.FS, 2048, 16384, 4
    x = synth.batch_traces(0, [0])
    f1, f2 = 0.2e12, 2.5e12
    out = O.zoom(x, fs, f1, f2, d, O.design_lowpass(63, d), n_fft)[0]
    grid = O.zoom_grid(fs, f1, f2, d, n_fft)
    inband = np.abs(grid - 0.5 * (f1 + f2)) < 0.5 * fs / d * 0.6
    sel = np.nonzero(inband)[0]
    ref = O.czt_bins(x, fs, grid[0], grid[-1], grid.size, sel)[0]
    # the filter is linear phase: compare magnitudes
    assert rel(np.abs(out[sel]), np.abs(ref)) < 5e-3


# ------------------------------------------------------------ helpers ------

def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_printed_fft_resolutions():
    g = golden()
    for key in ("fft_resolution_500_samples", "fft_resolution_250_samples"):
        e = g[key]
        assert O.fft_resolution(1.0 / e["ts_s"], e["n"]) == pytest.approx(e["delta_f_hz"], rel=1e-12)


def test_printed_zoom_resolution_equals_fft():
    g = golden()
    for key in ("zoom_resolution_equals_fft_500_samples", "zoom_resolution_equals_fft_250_samples"):
        e = g[key]
        fs = 1.0 / e["ts_s"]
        grid = O.zoom_grid(fs, 0.5e12, 1.5e12, 2, e["n"])
        assert np.diff(grid) == pytest.approx(e["delta_f_hz"], rel=1e-9)


def test_printed_two_tone_czt_resolution():
    e = golden()["czt_two_tone_resolution"]
    v = O.czt_resolution_eq24(e["f1_hz"], e["f2_hz"], e["m"])
    assert round(v, e["printed_decimals"]) == e["delta_f_hz"]
    # the same grid under this library's (M - 1) convention: pass
    # f2' = f1 + (f2 - f1)(M - 1)/M to get the paper's spacing
    f2p = e["f1_hz"] + (e["f2_hz"] - e["f1_hz"]) * (e["m"] - 1) / e["m"]
    assert O.czt_step(e["f1_hz"], f2p, e["m"]) == pytest.approx(v, rel=1e-12)


@pytest.mark.parametrize("fs,n_fft,delta", [(10e12, 500, 5e9), (8000.0, 128, 10.0), (20e12, 2048, 1e8)])
def test_zeros_for_delta_round_trip(fs, n_fft, delta):
    x = O.zeros_for_delta(fs, n_fft, delta)
    assert fs / n_fft - fs / (n_fft + x) >= delta * (1 - 1e-12)
    assert x == 0 or fs / n_fft - fs / (n_fft + x - 1) < delta


def test_zeros_for_delta_printed_case():
    # 500 samples at 10 THz (20 GHz); halving the spacing to 10 GHz needs
    # 500 appended zeros: 20 GHz - 10 THz/1000 = 10 GHz.
    assert O.zeros_for_delta(10e12, 500, 10e9) == 500


def test_m_for_resolution_matches_fft_spacing():
    # Eq. 25: M = (f2 - f1)/fs N_FFT gives the FFT spacing under Eq. 24.
    fs, f1, f2, n_fft = 10e12, 0.0, 2.5e12, 500
    m = O.m_for_resolution(fs, f1, f2, n_fft)
    assert m == 125
    assert O.czt_resolution_eq24(f1, f2, m) == pytest.approx(O.fft_resolution(fs, n_fft))


@pytest.mark.parametrize("taps,d", [(63, 4), (31, 2), (127, 16), (255, 64), (64, 3)])
def test_design_lowpass_matches_library_firwin(taps, d):
    # scipy's firwin: windowed sinc, cutoff 1/D of Nyquist, Hamming window,
    # unit DC gain; the oracle scales to DC gain D.
    ref = d * sps.firwin(taps, 1.0 / d, window="hamming")
    assert np.max(np.abs(O.design_lowpass(taps, d) - ref)) < 1e-13


def test_alias_identity_catches_planted_mix_sign(monkeypatch):
    # Plant a plausible mistake in the oracle (up-shift instead of down-shift)
    # and check that the alias-identity pin rejects it.
    n, d, taps, n_fft = 256, 4, 31, 2048
    fs, f1, f2 = 20e12, 0.9e12, 1.7e12
    x = rnd(n, 9)
    h = np.random.default_rng(10).standard_normal(taps)
    good = O.zoom(x, fs, f1, f2, d, h, n_fft)[0]
    orig = O._cycles_to_unit
    monkeypatch.setattr(O, "_cycles_to_unit", lambda cyc, sign: orig(cyc, -sign))
    bad = O.zoom(x, fs, f1, f2, d, h, n_fft)[0]
    assert rel(bad, good) > 0.1
