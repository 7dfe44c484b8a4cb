"""ctypes binding of ``libspec.so`` (declared in ``include/spec.h``).

Argument marshalling only: every transform step runs in the CUDA library.
Functions carry the C names.  Inputs may be CUDA torch tensors (device
path, asynchronous on the current torch stream), or numpy arrays / CPU
tensors (host path: the library stages them and returns when the output is
written).  Outputs are complex64 with the same residency as the input unless
``out`` is given.

If the library is missing, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspec.so")

SPEC_OK, SPEC_EINVAL, SPEC_ENOMEM, SPEC_ECUDA, SPEC_EUNSUPPORTED, SPEC_ETIMEOUT = range(6)
SPEC_CZT_AUTO, SPEC_CZT_BLUESTEIN, SPEC_CZT_GEMM_F16X3, SPEC_CZT_GEMM_F16X1, SPEC_CZT_GEMM_BF16X1 = 0, 1, 2, 3, 4

_STATUS = {SPEC_EINVAL: "SPEC_EINVAL", SPEC_ENOMEM: "SPEC_ENOMEM", SPEC_ECUDA: "SPEC_ECUDA",
           SPEC_EUNSUPPORTED: "SPEC_EUNSUPPORTED", SPEC_ETIMEOUT: "SPEC_ETIMEOUT"}

EXPORTS = ("spec_ctx_create", "spec_ctx_destroy", "spec_last_error", "spec_ctx_check",
           "spec_selftest_wait_timeout", "spec_measure_fp32_peak",
           "spec_fft", "spec_czt", "spec_czt_spiral", "spec_zoom", "spec_czt_static", "spec_ragged",
           "spec_ragged_launches", "spec_ragged_plan_info", "spec_czt_auto_mode", "spec_tune_cache_store", "spec_tune_cache_lookup",
           "spec_zeros_for_delta", "spec_m_for_resolution", "spec_design_lowpass")

SPEC_KIND_FFT, SPEC_KIND_CZT, SPEC_KIND_ZOOM = 0, 1, 2


class spec_desc(C.Structure):
    """One trace of a ragged batch (include/spec.h)."""
    _fields_ = [("x_off", C.c_int64), ("n", C.c_int64), ("out_off", C.c_int64), ("f1", C.c_double),
                ("f2", C.c_double), ("n_fft", C.c_int64), ("m", C.c_int64), ("d", C.c_int64),
                ("taps_off", C.c_int64), ("n_taps", C.c_int64)]


_lib = None


class SpecError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load libspec.so once (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    i64, dbl, vp, fp = C.c_int64, C.c_double, C.c_void_p, C.c_void_p
    L.spec_ctx_create.argtypes = [C.POINTER(vp), C.c_int]
    L.spec_ctx_create.restype = C.c_int
    L.spec_ctx_destroy.argtypes = [vp]
    L.spec_ctx_destroy.restype = None
    L.spec_last_error.argtypes = [vp]
    L.spec_last_error.restype = C.c_char_p
    L.spec_ctx_check.argtypes = [vp, vp]
    L.spec_ctx_check.restype = C.c_int
    L.spec_measure_fp32_peak.argtypes = [vp, C.POINTER(dbl), vp]
    L.spec_measure_fp32_peak.restype = C.c_int
    L.spec_selftest_wait_timeout.argtypes = [vp, i64, vp]
    L.spec_selftest_wait_timeout.restype = C.c_int
    L.spec_fft.argtypes = [vp, fp, i64, i64, i64, dbl, i64, fp, i64, vp]
    L.spec_fft.restype = C.c_int
    L.spec_czt.argtypes = [vp, fp, i64, i64, i64, dbl, dbl, dbl, i64, C.c_int, fp, i64, vp]
    L.spec_czt.restype = C.c_int
    L.spec_czt_spiral.argtypes = [vp, fp, i64, i64, i64, dbl, dbl, dbl, i64, dbl, dbl, fp, i64, vp]
    L.spec_czt_spiral.restype = C.c_int
    L.spec_zoom.argtypes = [vp, fp, i64, i64, i64, dbl, dbl, dbl, i64, fp, i64, i64, fp, i64, vp]
    L.spec_zoom.restype = C.c_int
    L.spec_ragged.argtypes = [vp, C.c_int, C.POINTER(spec_desc), i64, dbl, fp, fp, fp, vp]
    L.spec_ragged.restype = C.c_int
    L.spec_ragged_launches.argtypes = [vp, C.c_int, C.POINTER(spec_desc), i64, dbl]
    L.spec_ragged_launches.restype = i64
    L.spec_czt_static.argtypes = [fp, i64, i64, i64, dbl, dbl, dbl, i64, fp, i64, vp]
    L.spec_czt_static.restype = C.c_int
    L.spec_ragged_plan_info.argtypes = [vp, C.c_int, C.POINTER(spec_desc), i64, dbl, C.POINTER(C.c_float),
                                        C.POINTER(C.c_float)]
    L.spec_ragged_plan_info.restype = C.c_int
    L.spec_czt_auto_mode.argtypes = [vp, i64, i64, dbl, dbl, dbl, i64, C.POINTER(C.c_int), vp]
    L.spec_czt_auto_mode.restype = C.c_int
    L.spec_tune_cache_store.argtypes = [C.c_char_p, C.c_char_p, C.c_char_p, C.c_char_p]
    L.spec_tune_cache_store.restype = C.c_int
    L.spec_tune_cache_lookup.argtypes = [C.c_char_p, C.c_char_p, C.c_char_p, C.c_char_p, C.c_int]
    L.spec_tune_cache_lookup.restype = C.c_int
    L.spec_zeros_for_delta.argtypes = [dbl, i64, dbl]
    L.spec_zeros_for_delta.restype = i64
    L.spec_m_for_resolution.argtypes = [dbl, dbl, dbl, i64]
    L.spec_m_for_resolution.restype = i64
    L.spec_design_lowpass.argtypes = [fp, i64, i64]
    L.spec_design_lowpass.restype = C.c_int
    _lib = L
    return L


class Context:
    """Owns one ``spec_ctx`` (tables, caches, staging) on a CUDA device."""

    def __init__(self, device: int = 0):
        L = lib()
        h = C.c_void_p()
        st = L.spec_ctx_create(C.byref(h), int(device))
        if st != SPEC_OK:
            raise SpecError(st, L.spec_last_error(None).decode())
        self.handle = h
        self.device = int(device)

    def close(self):
        if self.handle:
            lib().spec_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def check(self, status):
        if status != SPEC_OK:
            raise SpecError(status, lib().spec_last_error(self.handle).decode())

    def sync(self, stream=None):
        self.check(lib().spec_ctx_check(self.handle, stream))


# ---------------------------------------------------------------- marshal ---

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _rows(x):
    """(pointer, batch, row stride, device?, stream) of a float32 [batch, n] input."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.float32:
            raise TypeError("x must be float32")
        if x.dim() == 1:
            x = x.unsqueeze(0)
        if x.dim() != 2 or (x.shape[1] > 1 and x.stride(1) != 1):
            raise ValueError("x must be [batch, n] with unit column stride")
        dev = x.is_cuda
        stream = torch.cuda.current_stream(x.device).cuda_stream if dev else None
        return x, x.data_ptr(), x.shape[0], x.stride(0) if x.shape[0] > 1 else x.shape[1], dev, stream
    a = np.asarray(x)
    if a.dtype != np.float32:
        raise TypeError("x must be float32")
    if a.ndim == 1:
        a = a[None, :]
    if a.ndim != 2 or (a.shape[1] > 1 and a.strides[1] != 4):
        raise ValueError("x must be [batch, n] with unit column stride")
    ld = a.strides[0] // 4 if a.shape[0] > 1 else a.shape[1]
    return a, a.ctypes.data, a.shape[0], ld, False, None


def _out(like_dev, x, batch, bins, out):
    if out is not None:
        if _is_torch(out):
            import torch
            if out.dtype != torch.complex64 or out.dim() != 2 or out.stride(1) != 1:
                raise ValueError("out must be complex64 [batch, >= bins] with unit column stride")
            return out, out.data_ptr(), out.stride(0) if out.shape[0] > 1 else out.shape[1]
        if out.dtype != np.complex64 or out.ndim != 2 or out.strides[1] != 8:
            raise ValueError("out must be complex64 [batch, >= bins] with unit column stride")
        return out, out.ctypes.data, out.strides[0] // 8 if out.shape[0] > 1 else out.shape[1]
    if like_dev:
        import torch
        o = torch.empty((batch, bins), dtype=torch.complex64, device=x.device)
        return o, o.data_ptr(), bins
    o = np.empty((batch, bins), dtype=np.complex64)
    return o, o.ctypes.data, bins


def _taps_ptr(taps):
    if _is_torch(taps):
        import torch
        if taps.dtype != torch.float32 or not taps.is_contiguous():
            raise TypeError("taps must be contiguous float32")
        return taps, taps.data_ptr(), taps.numel()
    t = np.ascontiguousarray(taps, dtype=np.float32)
    return t, t.ctypes.data, t.size


# ------------------------------------------------------------- transforms ---

def spec_fft(ctx: Context, x, fs: float, n_fft: int, n: int | None = None, out=None, stream=None):
    """Zero-padded FFT: N_FFT/2 + 1 bins per trace (Section 2.1, Eq. 2-3)."""
    keep, px, batch, ld_x, dev, st = _rows(x)
    n = keep.shape[1] if n is None else int(n)
    o, po, ld_o = _out(dev, keep, batch, n_fft // 2 + 1, out)
    ctx.check(lib().spec_fft(ctx.handle, px, batch, n, ld_x, float(fs), int(n_fft), po, ld_o,
                             st if stream is None else stream))
    return o


def spec_czt(ctx: Context, x, fs: float, f1: float, f2: float, m: int, n: int | None = None,
             mode: int = SPEC_CZT_AUTO, out=None, stream=None):
    """Chirp-z transform at M points f1 .. f2 inclusive (Section 2.3, Eq. 11-23)."""
    keep, px, batch, ld_x, dev, st = _rows(x)
    n = keep.shape[1] if n is None else int(n)
    o, po, ld_o = _out(dev, keep, batch, int(m), out)
    ctx.check(lib().spec_czt(ctx.handle, px, batch, n, ld_x, float(fs), float(f1), float(f2), int(m),
                             int(mode), po, ld_o, st if stream is None else stream))
    return o


def spec_czt_spiral(ctx: Context, x, fs: float, f1: float, f2: float, m: int, a0: float, w0: float,
                    n: int | None = None, out=None, stream=None):
    """Chirp-z on the spiral z_k = A W^{-k}, A = a0 e^{j2pi f1/fs}, W = w0 e^{-j2pi step/fs}
    (Section 2.3, Eq. 11 with Eq. 16-17)."""
    keep, px, batch, ld_x, dev, st = _rows(x)
    n = keep.shape[1] if n is None else int(n)
    o, po, ld_o = _out(dev, keep, batch, int(m), out)
    ctx.check(lib().spec_czt_spiral(ctx.handle, px, batch, n, ld_x, float(fs), float(f1), float(f2), int(m),
                                    float(a0), float(w0), po, ld_o, st if stream is None else stream))
    return o


def spec_zoom(ctx: Context, x, fs: float, f1: float, f2: float, d: int, taps, n_fft: int,
              n: int | None = None, out=None, stream=None):
    """Zoom FFT: N_FFT/D bins around (f1 + f2)/2 (Section 2.2, Eq. 6-10)."""
    keep, px, batch, ld_x, dev, st = _rows(x)
    n = keep.shape[1] if n is None else int(n)
    tk, pt, nt = _taps_ptr(taps)
    o, po, ld_o = _out(dev, keep, batch, int(n_fft) // int(d), out)
    ctx.check(lib().spec_zoom(ctx.handle, px, batch, n, ld_x, float(fs), float(f1), float(f2), int(d),
                              pt, nt, int(n_fft), po, ld_o, st if stream is None else stream))
    return o


def spec_ragged(ctx: Context, kind: int, descs, fs: float, x_pool, X_pool, taps_pool=None, stream=None):
    """Ragged batch: descs is a sequence of spec_desc (or dicts of its fields),
    or an array from ``desc_array`` (passed through without copying: build it
    once for a batch that is transformed repeatedly); pools are CUDA tensors
    (x float32, X complex64, taps float32)."""
    import torch
    arr, n = _desc_array(descs)
    st = torch.cuda.current_stream(x_pool.device).cuda_stream if stream is None else stream
    ctx.check(lib().spec_ragged(ctx.handle, int(kind), arr, n, float(fs), x_pool.data_ptr(),
                                taps_pool.data_ptr() if taps_pool is not None else None,
                                X_pool.data_ptr(), st))
    return X_pool


class DescArray:
    """A ctypes array of spec_desc built once (see desc_array)."""

    def __init__(self, descs):
        n = len(descs)
        self.arr = (spec_desc * max(1, n))()
        for i, dsc in enumerate(descs):
            self.arr[i] = dsc if isinstance(dsc, spec_desc) else spec_desc(**dsc)
        self.n = n

    def __len__(self):
        return self.n


def desc_array(descs) -> DescArray:
    """Marshal a descriptor list once, for repeated spec_ragged calls."""
    return DescArray(descs)


def _desc_array(descs):
    if isinstance(descs, DescArray):
        return descs.arr, descs.n
    d = DescArray(descs)
    return d.arr, d.n


def spec_ragged_launches(ctx: Context, kind: int, descs, fs: float) -> int:
    arr, n = _desc_array(descs)
    return int(lib().spec_ragged_launches(ctx.handle, int(kind), arr, n, float(fs)))


def spec_czt_auto_mode(ctx: Context, batch: int, n: int, fs: float, f1: float, f2: float, m: int,
                       stream=None) -> int:
    """The explicit mode SPEC_CZT_AUTO stands for at (batch, n, m)."""
    out = C.c_int(0)
    ctx.check(lib().spec_czt_auto_mode(ctx.handle, int(batch), int(n), float(fs), float(f1), float(f2), int(m),
                                       C.byref(out), _stream_handle(stream)))
    return out.value


def spec_tune_cache_store(path: str, device: str, key: str, value: str) -> int:
    return int(lib().spec_tune_cache_store(path.encode(), device.encode(), key.encode(), value.encode()))


def spec_tune_cache_lookup(path: str, device: str, key: str):
    """The cached value, or None."""
    buf = C.create_string_buffer(256)
    found = lib().spec_tune_cache_lookup(path.encode(), device.encode(), key.encode(), buf, 256)
    return buf.value.decode() if found else None


def spec_ragged_plan_info(ctx: Context, kind: int, descs, fs: float):
    """(uses the work queue?, queue us, per-shape us) of the cached plan, or None."""
    arr, n = _desc_array(descs)
    tq, tc = C.c_float(0.0), C.c_float(0.0)
    r = int(lib().spec_ragged_plan_info(ctx.handle, int(kind), arr, n, float(fs), C.byref(tq), C.byref(tc)))
    return None if r < 0 else (bool(r), tq.value, tc.value)


# ---------------------------------------------------------------- helpers ---

def spec_zeros_for_delta(fs: float, n_fft: int, delta: float) -> int:
    return int(lib().spec_zeros_for_delta(float(fs), int(n_fft), float(delta)))


def spec_m_for_resolution(fs: float, f1: float, f2: float, n_fft: int) -> int:
    return int(lib().spec_m_for_resolution(float(fs), float(f1), float(f2), int(n_fft)))


def spec_design_lowpass(n_taps: int, d: int) -> np.ndarray:
    out = np.empty(int(n_taps), dtype=np.float32)
    st = lib().spec_design_lowpass(out.ctypes.data, int(n_taps), int(d))
    if st != SPEC_OK:
        raise SpecError(st, "invalid n_taps or d")
    return out


# ------------------------------------------------------- status, self-test ---

def _stream_handle(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def ctx_status(ctx: Context, stream=None) -> int:
    """spec_ctx_check's raw status (SPEC_OK, SPEC_ETIMEOUT, ...) without raising."""
    return lib().spec_ctx_check(ctx.handle, _stream_handle(stream))


def spec_selftest_wait_timeout(ctx: Context, timeout_us: int, stream=None):
    """Launch the bounded-wait self-test; the next ctx_status is SPEC_ETIMEOUT."""
    ctx.check(lib().spec_selftest_wait_timeout(ctx.handle, int(timeout_us), _stream_handle(stream)))


def spec_measure_fp32_peak(ctx: Context, stream=None) -> float:
    """Measured FP32 FMA throughput of the context's device, TFLOP/s."""
    out = C.c_double(0.0)
    ctx.check(lib().spec_measure_fp32_peak(ctx.handle, C.byref(out), _stream_handle(stream)))
    return out.value
