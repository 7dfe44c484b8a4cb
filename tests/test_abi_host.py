"""The C-ABI library builds, loads and exports every declared symbol; host
helpers agree with the oracle; argument errors come back before any launch.
CPU only (no kernel runs)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import spec_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spec.h")


@pytest.fixture(scope="module")
def spec():
    from paper_2108_03948_gb300 import build as b
    try:
        b.build()
    except RuntimeError as e:          # no nvcc on this machine
        pytest.skip(f"cannot build the CUDA library here: {e}")
    from paper_2108_03948_gb300 import spec as s
    s.lib()
    return s


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SPEC_API\s+[\w\s\*]+?\b(spec_\w+)\s*\(", text)))


def test_header_declares_the_paper_entry_points():
    syms = declared_symbols()
    for name in ("spec_fft", "spec_czt", "spec_zoom"):
        assert name in syms


def test_library_exports_every_declared_symbol(spec):
    lib = spec.lib()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", spec.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (spec_\w+)", out))
    assert set(declared_symbols()) <= exported
    # nothing but the ABI is exported under the spec_ prefix
    assert exported <= set(declared_symbols())


def test_binding_names_match_header(spec):
    assert set(spec.EXPORTS) == set(declared_symbols())


@pytest.mark.parametrize("fs,n_fft,delta", [(10e12, 500, 5e9), (10e12, 500, 10e9), (8000.0, 128, 10.0),
                                            (20e12, 2048, 1e8), (1.0, 7, 0.0)])
def test_zeros_for_delta_matches_oracle(spec, fs, n_fft, delta):
    assert spec.spec_zeros_for_delta(fs, n_fft, delta) == O.zeros_for_delta(fs, n_fft, delta)


def test_zeros_for_delta_rejects(spec):
    assert spec.spec_zeros_for_delta(10e12, 500, 20e9) == -1      # delta >= fs/N
    assert spec.spec_zeros_for_delta(-1.0, 500, 1.0) == -1


@pytest.mark.parametrize("fs,f1,f2,n_fft", [(10e12, 0.0, 2.5e12, 500), (20e12, 0.2e12, 2.5e12, 16384),
                                            (8000.0, 100.0, 1000.0, 128), (20e12, 1e12, 0.5e12, 4096)])
def test_m_for_resolution_matches_oracle(spec, fs, f1, f2, n_fft):
    assert spec.spec_m_for_resolution(fs, f1, f2, n_fft) == O.m_for_resolution(fs, f1, f2, n_fft)


@pytest.mark.parametrize("taps,d", [(63, 4), (31, 2), (127, 16), (255, 64), (1, 1), (10, 3)])
def test_design_lowpass_matches_oracle(spec, taps, d):
    got = spec.spec_design_lowpass(taps, d)
    ref = O.design_lowpass(taps, d)
    assert np.max(np.abs(got - ref)) <= 2e-7 * max(1.0, np.max(np.abs(ref)))


def test_null_context_is_rejected_before_any_cuda_call(spec):
    lib = spec.lib()
    x = np.zeros(16, np.float32)
    X = np.zeros(9, np.complex64)
    assert lib.spec_fft(None, x.ctypes.data, 1, 16, 16, 1.0, 16, X.ctypes.data, 9, None) == spec.SPEC_EINVAL
    assert lib.spec_czt(None, x.ctypes.data, 1, 16, 16, 1.0, 0.0, 0.5, 9, 0, X.ctypes.data, 9,
                        None) == spec.SPEC_EINVAL
    assert lib.spec_zoom(None, x.ctypes.data, 1, 16, 16, 1.0, 0.0, 0.5, 1, x.ctypes.data, 1, 16,
                         X.ctypes.data, 16, None) == spec.SPEC_EINVAL
    assert lib.spec_design_lowpass(None, 5, 2) == spec.SPEC_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2108_03948_gb300 import spec as s
    monkeypatch.setattr(s, "_lib", None)
    monkeypatch.setattr(s, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError):
        s.lib()


def test_context_without_gpu_reports_an_error(spec):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(spec.SpecError):
        spec.Context(0)
