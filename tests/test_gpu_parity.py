"""Parity of the CUDA transforms with the FP64 oracle, element by element on
the same seeded float32 inputs: relative L2 error <= 1e-5 per spectrum (the
accuracy bar of the FP32 paths).  Sizes span several CTA tiles, clusters and
ragged tails; the full-size batch runs in the bench's launch configuration
and is checked on sampled traces."""
import numpy as np
import pytest

from oracle import spec_oracle as O
from paper_2108_03948_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_2108_03948_gb300 import build
    build.build()
    from paper_2108_03948_gb300 import spec
    c = spec.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def S():
    from paper_2108_03948_gb300 import spec
    return spec


def rel_rows(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    return np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)


def traces(batch, n, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((batch, n)).astype(np.float32)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------------- FFT ------

FFT_CASES = [
    (3, 2048, 16384), (5, 2047, 16384), (4, 1000, 8192), (3, 4097, 65536), (2, 8192, 65536),
    (2, 16384, 131072), (2, 4096, 4096), (3, 1, 1), (3, 1, 2), (3, 2, 2), (2, 3, 4), (2, 5, 8),
    (2, 16, 16), (2, 17, 32), (3, 33, 64), (7, 100, 128), (9, 300, 512), (5, 31, 4096), (3, 6000, 8192),
]


# traces that need a cluster of 2-8 CTAs (R LZ/8192 of them): every (LZ, R)
# of the cluster kernel, full and partial traces
FFT_CASES += [(2, 4000, 32768), (2, 8000, 32768), (2, 2000, 32768), (2, 1500, 65536), (2, 3000, 65536),
              (1, 5000, 131072), (2, 1025, 65536), (3, 2049, 65536)]


# N_FFT not a power of two (the resolution fs/N_FFT of Eq. 3 chosen freely):
# the chirp-z on the DFT grid; the paper's unpadded 500-sample trace among them
FFT_CASES += [(3, 500, 500), (2, 500, 1000), (2, 2048, 20000), (3, 1000, 12345), (2, 7, 9), (3, 100, 101),
              (2, 20000, 40000)]
# even lengths whose half has only the factors 2, 3, 5, 7 run the mixed-radix
# padded FFT (the sweep's 2^k 5^j lengths; radix 3 and 7 passes; R = 1 and a
# one-point residue DFT)
FFT_CASES += [(4, 500, 2000), (3, 500, 10000), (2, 500, 20000), (3, 1000, 2000), (2, 2000, 26000),
              (5, 333, 1050), (3, 12, 42), (2, 1, 6), (3, 4000, 26460)]


@pytest.mark.parametrize("batch,n,n_fft", FFT_CASES)
def test_fft_parity(ctx, S, batch, n, n_fft):
    x = traces(batch, n, 100 + n)
    got = S.spec_fft(ctx, dev(x), 20e12, n_fft).cpu().numpy()
    assert got.shape == (batch, n_fft // 2 + 1)
    err = rel_rows(got, O.fft_padded(x, n_fft))
    assert err.max() <= TOL, err


def test_fft_thz_traces_and_strides(ctx, S):
    x = synth.batch_traces(1, range(6))
    base = torch.zeros((6, 2100), dtype=torch.float32, device="cuda")
    base[:, :2048] = dev(x)
    out = torch.full((6, 8300), float("nan"), dtype=torch.complex64, device="cuda")
    S.spec_fft(ctx, base, 20e12, 16384, n=2048, out=out)
    got = out[:, :8193].cpu().numpy()
    assert rel_rows(got, O.fft_padded(x, 16384)).max() <= TOL
    assert torch.isnan(out[:, 8193:].real).all()        # padding columns untouched


def test_fft_full_traces_at_odd_row_starts(ctx, S):
    """Full traces (n = 2 LZ) load their packed samples as 8-byte pairs when
    the row starts on an 8-byte boundary and as two 4-byte loads otherwise:
    an odd row stride (2051) alternates the two cases row by row, and a base
    offset by one float swaps them."""
    x = traces(6, 2048, 77)
    ref = O.fft_padded(x, 16384)
    for off in (0, 1):
        base = torch.zeros((6 * 2051 + 1,), dtype=torch.float32, device="cuda")
        rows = base[off:off + 6 * 2051].view(6, 2051)
        rows[:, :2048] = dev(x)
        got = S.spec_fft(ctx, rows, 20e12, 16384, n=2048).cpu().numpy()
        assert rel_rows(got, ref).max() <= TOL, off


# ---------------------------------------------------------------- CZT ------

CZT_CASES = [
    (3, 2048, 0.2e12, 2.5e12, 1024), (4, 1000, 0.1e12, 3.6e12, 256), (2, 1024, 0.8e12, 1.2e12, 512),
    (3, 2048, 2.5e12, 0.2e12, 1024), (2, 500, 1.0e12, 1.0e12, 1), (3, 8192, 0.3e12, 3.0e12, 4096),
    (2, 1, 0.5e12, 1.0e12, 1), (2, 3, 0.5e12, 1.0e12, 5), (5, 333, -2e12, 9.9e12, 77), (2, 64, 0.0, 19.6875e12, 64),
    (1, 2048, 0.2e12, 2.5e12, 1024), (7, 4000, 0.3e12, 1.3e12, 4000),
]


@pytest.mark.parametrize("batch,n,f1,f2,m", CZT_CASES)
def test_czt_parity(ctx, S, batch, n, f1, f2, m):
    fs = 20e12
    x = traces(batch, n, 200 + n + m)
    got = S.spec_czt(ctx, dev(x), fs, f1, f2, m).cpu().numpy()
    assert got.shape == (batch, m)
    err = rel_rows(got, O.czt(x, fs, f1, f2, m))
    assert err.max() <= TOL, err


def test_czt_table_cache_reuse_and_thz(ctx, S):
    fs = 20e12
    x = synth.batch_traces(1, range(4))
    a = S.spec_czt(ctx, dev(x), fs, 0.2e12, 2.5e12, 1024).cpu().numpy()
    b = S.spec_czt(ctx, dev(x), fs, 0.2e12, 2.5e12, 1024).cpu().numpy()
    assert np.array_equal(a, b)
    assert rel_rows(a, O.czt(x, fs, 0.2e12, 2.5e12, 1024)).max() <= TOL


# --------------------------------------------------------------- Zoom ------

ZOOM_CASES = [
    (3, 2048, 0.2e12, 2.5e12, 4, 63, 16384), (2, 2048, 1.0e12, 1.7e12, 1, 1, 4096),
    (3, 8192, 0.5e12, 1.5e12, 16, 127, 65536), (2, 8192, 0.5e12, 1.5e12, 4, 31, 65536),
    (4, 30, 0.5e12, 1.5e12, 2, 5, 64), (3, 1000, 0.1e12, 2.0e12, 8, 45, 8192), (2, 2047, 3e12, 4e12, 2, 64, 16384),
    (1, 2048, 0.2e12, 2.5e12, 4, 63, 16384), (5, 3000, 0.2e12, 0.9e12, 3, 40, 24576),
    # L_out above K/4 with 16-byte staging loads (D = 4): the FFT's full first pass;
    # K = 512 with L_out <= K/4 (sparse first pass, one warp per trace)
    (3, 4096, 0.5e12, 1.5e12, 4, 63, 8192), (3, 400, 0.5e12, 1.5e12, 4, 31, 2048),
    # FIR kernel + pruned cluster FFT: K = 32768 (4-CTA cluster), a 100 k-sample trace,
    # the long-trace shape (262144 samples, D = 64, 255 taps, K = 32768), D not a power of two
    (3, 8000, 0.5e12, 2.5e12, 2, 101, 65536), (2, 100000, 0.3e12, 0.4e12, 64, 255, 262144),
    (2, 262144, 0.3e12, 0.4e12, 64, 255, 1 << 21), (2, 70000, 1.0e12, 1.2e12, 48, 200, 196608),
]


@pytest.mark.parametrize("batch,n,f1,f2,d,nt,n_fft", ZOOM_CASES)
def test_zoom_parity(ctx, S, batch, n, f1, f2, d, nt, n_fft):
    fs = 20e12
    x = traces(batch, n, 300 + n + d)
    h = O.design_lowpass(nt, d).astype(np.float32)
    got = S.spec_zoom(ctx, dev(x), fs, f1, f2, d, dev(h), n_fft).cpu().numpy()
    assert got.shape == (batch, n_fft // d)
    err = rel_rows(got, O.zoom(x, fs, f1, f2, d, h, n_fft))
    assert err.max() <= TOL, err


# ------------------------------------------------------ host-buffer path ---

def test_host_buffers_match_device_path(ctx, S):
    cfg = synth.UNIFORM[0]
    x = synth.batch_traces(1, range(5))
    h = O.design_lowpass(cfg.zoom_taps, cfg.zoom_d).astype(np.float32)
    for f_host, f_dev in [
        (lambda: S.spec_fft(ctx, x, cfg.fs, cfg.n_fft), lambda: S.spec_fft(ctx, dev(x), cfg.fs, cfg.n_fft)),
        (lambda: S.spec_czt(ctx, x, cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m),
         lambda: S.spec_czt(ctx, dev(x), cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m)),
        (lambda: S.spec_zoom(ctx, x, cfg.fs, cfg.zoom_f1, cfg.zoom_f2, cfg.zoom_d, h, cfg.zoom_n_fft),
         lambda: S.spec_zoom(ctx, dev(x), cfg.fs, cfg.zoom_f1, cfg.zoom_f2, cfg.zoom_d, dev(h), cfg.zoom_n_fft)),
    ]:
        a = f_host()
        b = f_dev().cpu().numpy()
        assert isinstance(a, np.ndarray)
        assert np.array_equal(a, b)


def test_host_pipeline_chunks_match_device_path(ctx, S):
    """Host buffers above 16 MiB of traffic run in overlapped chunks of
    traces (4001 traces: a ragged last chunk).  Every chunk runs the same
    kernels per trace as the device-pointer call, so the spectra are
    bit-identical: pageable and pinned memory, either direction staged alone,
    and strided rows on both sides."""
    cfg = synth.UNIFORM[1]
    B = 4001
    x = traces(B, cfg.n, 11)
    xd = dev(x)
    h = O.design_lowpass(cfg.zoom_taps, cfg.zoom_d).astype(np.float32)
    calls = {
        "fft": (cfg.n_fft // 2 + 1, lambda a, **k: S.spec_fft(ctx, a, cfg.fs, cfg.n_fft, **k)),
        "czt": (cfg.czt_m, lambda a, **k: S.spec_czt(ctx, a, cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m, **k)),
        "zoom": (cfg.zoom_n_fft // cfg.zoom_d,
                 lambda a, **k: S.spec_zoom(ctx, a, cfg.fs, cfg.zoom_f1, cfg.zoom_f2, cfg.zoom_d, h, cfg.zoom_n_fft,
                                            **k)),
    }
    xp = torch.from_numpy(x).pin_memory()
    wide = np.zeros((B, cfg.n + 5), dtype=np.float32)
    wide[:, :cfg.n] = x
    for name, (bins, f) in calls.items():
        ref = f(xd).cpu().numpy()
        assert np.array_equal(f(x), ref), name                                  # pageable in and out
        op = torch.empty((B, bins), dtype=torch.complex64).pin_memory()
        f(xp, out=op)
        assert np.array_equal(op.numpy(), ref), name                           # pinned in and out
        od = torch.empty((B, bins), dtype=torch.complex64, device="cuda")
        f(x, out=od)
        assert np.array_equal(od.cpu().numpy(), ref), name                     # host in, device out
        oh = np.zeros((B, bins + 3), dtype=np.complex64)
        f(xd, out=oh[:, :bins])
        assert np.array_equal(oh[:, :bins], ref), name                         # device in, host out
        assert not oh[:, bins:].any(), name                                     # padding columns untouched
        ow = np.zeros((B, bins + 3), dtype=np.complex64)
        f(wide[:, :cfg.n], out=ow[:, :bins])
        assert np.array_equal(ow[:, :bins], ref), name                         # strided host rows


def test_host_buffers_rejected_before_any_copy(ctx, S):
    """A host-buffer call with a bad argument returns SPEC_EINVAL before the
    pipeline starts: the caller's output buffer is untouched."""
    lib = S.lib()
    x = np.ones((3, 64), dtype=np.float32)
    X = np.full((3, 64), 7 + 7j, dtype=np.complex64)
    px, pX = x.ctypes.data, X.ctypes.data
    E = S.SPEC_EINVAL
    assert lib.spec_fft(ctx.handle, px, 3, 64, 64, 1.0, 1 << 25, pX, 64, None) == E          # n_fft
    assert lib.spec_czt(ctx.handle, px, 3, 64, 64, 1.0, 0.0, 0.4, 8, 9, pX, 64, None) == E    # mode
    assert lib.spec_zoom(ctx.handle, px, 3, 64, 64, 1.0, 0.1, 0.2, 3, px, 8, 64, pX, 64, None) == E  # d
    assert (X == 7 + 7j).all()


# --------------------------------------------------------------- errors ----

def test_invalid_arguments_return_einval(ctx, S):
    lib = S.lib()
    x = torch.zeros((2, 64), device="cuda")
    X = torch.zeros((2, 64), dtype=torch.complex64, device="cuda")
    px, pX = x.data_ptr(), X.data_ptr()
    E = S.SPEC_EINVAL
    assert lib.spec_fft(ctx.handle, px, 2, 64, 64, 1.0, 1 << 25, pX, 64, None) == E  # n_fft above 2^24
    assert lib.spec_fft(ctx.handle, px, 2, 64, 64, 1.0, 32, pX, 64, None) == E       # n_fft < n
    assert lib.spec_fft(ctx.handle, px, 2, 64, 60, 1.0, 64, pX, 64, None) == E       # ld_x < n
    assert lib.spec_fft(ctx.handle, px, 2, 64, 64, 0.0, 64, pX, 64, None) == E       # fs
    assert lib.spec_fft(ctx.handle, px, 2, 64, 64, 1.0, 64, px, 64, None) == E       # overlap
    assert lib.spec_czt(ctx.handle, px, 2, 64, 64, 1.0, 0.0, 0.4, 0, 0, pX, 64, None) == E   # m
    assert lib.spec_czt(ctx.handle, px, 2, 64, 64, 1.0, 0.0, 0.4, 8, 9, pX, 64, None) == E   # mode
    assert lib.spec_czt(ctx.handle, px, 2, 64, 64, 1.0, float("nan"), 0.4, 8, 0, pX, 64, None) == E
    h = torch.ones(8, device="cuda")
    # L_out = ceil((64 + 7)/4) = 18 > K = 16
    assert lib.spec_zoom(ctx.handle, px, 2, 64, 64, 1.0, 0.1, 0.2, 4, h.data_ptr(), 8, 64, pX, 64, None) == E
    assert lib.spec_zoom(ctx.handle, px, 2, 64, 64, 1.0, 0.1, 0.2, 3, h.data_ptr(), 8, 64, pX, 64, None) == E
    assert b"n_fft" in lib.spec_last_error(ctx.handle) or lib.spec_last_error(ctx.handle)
    assert np.all(X.cpu().numpy() == 0)                 # nothing was written
    # an empty batch is a no-op
    assert lib.spec_fft(ctx.handle, px, 0, 64, 64, 1.0, 64, pX, 64, None) == S.SPEC_OK


# ------------------------------------------------- full-size workload 1 ---

def test_workload1_full_batch_sampled(ctx, S):
    cfg = synth.UNIFORM[1]
    x = synth.batch_traces(1, range(cfg.batch))
    xd = dev(x)
    h = O.design_lowpass(cfg.zoom_taps, cfg.zoom_d).astype(np.float32)
    X = S.spec_fft(ctx, xd, cfg.fs, cfg.n_fft)
    Z = S.spec_czt(ctx, xd, cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m)
    U = S.spec_zoom(ctx, xd, cfg.fs, cfg.zoom_f1, cfg.zoom_f2, cfg.zoom_d, dev(h), cfg.zoom_n_fft)
    torch.cuda.synchronize()
    pick = [0, 1, 1000, 2047, 4094, 4095]
    xs = x[pick]
    assert rel_rows(X[pick].cpu().numpy(), O.fft_padded(xs, cfg.n_fft)).max() <= TOL
    assert rel_rows(Z[pick].cpu().numpy(), O.czt(xs, cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m)).max() <= TOL
    assert rel_rows(U[pick].cpu().numpy(), O.zoom(xs, cfg.fs, cfg.zoom_f1, cfg.zoom_f2, cfg.zoom_d, h,
                                                  cfg.zoom_n_fft)).max() <= TOL
    assert torch.isfinite(torch.view_as_real(X)).all()
    assert torch.isfinite(torch.view_as_real(Z)).all()
    assert torch.isfinite(torch.view_as_real(U)).all()


# ------------------------------------- many clusters resident at once ------

@pytest.mark.parametrize("kind", ["fft65536", "fft32768", "zoom32768"])
def test_cluster_paths_under_full_occupancy(ctx, S, kind):
    # Transforms large enough to run on thread-block clusters stage their
    # result through peer shared memory; with thousands of clusters in flight
    # any missing cluster-wide barrier shows as corrupted rows.  The batch
    # repeats 8 distinct traces, so every copy must equal its original bit for
    # bit and the originals must match the oracle.
    n = 8192 if kind != "fft32768" else 4096
    base = traces(8, n, 77)
    x = np.tile(base, (150, 1))
    if kind.startswith("fft"):
        n_fft = int(kind[3:])
        got = S.spec_fft(ctx, dev(x), 20e12, n_fft).cpu().numpy()
        ref = O.fft_padded(base, n_fft)
    else:
        h = O.design_lowpass(63, 2).astype(np.float32)
        got = S.spec_zoom(ctx, dev(x), 20e12, 0.2e12, 3.0e12, 2, dev(h), 65536).cpu().numpy()
        ref = O.zoom(base, 20e12, 0.2e12, 3.0e12, 2, h, 65536)
    got = got.reshape(150, 8, -1)
    assert (got == got[:1]).all()
    assert rel_rows(got[0], ref).max() <= TOL


# ------------------------------------------------ the cluster FFT kernel ------

CLUSTER_CASES = [(2, 4000, 32768), (2, 8000, 32768), (2, 2000, 32768), (2, 1500, 65536), (2, 3000, 65536),
                 (1, 5000, 131072), (2, 1025, 65536), (3, 2049, 65536), (2, 8192, 65536), (2, 4096, 32768)]


def test_fft_cluster_kernel_parity(S, monkeypatch):
    # SPEC_FFT_CLUSTER=1 (read when a context is created) puts every (LZ, R)
    # the cluster kernel has an instance for on it: conjugate-paired residues,
    # spectrum assembled in the cluster's shared memory
    monkeypatch.setenv("SPEC_FFT_CLUSTER", "1")
    with S.Context(0) as c:
        for batch, n, n_fft in CLUSTER_CASES:
            x = traces(batch, n, n + n_fft)
            got = S.spec_fft(c, dev(x), 20e12, n_fft).cpu().numpy()
            err = rel_rows(got, O.fft_padded(x, n_fft))
            assert err.max() <= TOL, (batch, n, n_fft, err.max())


# every (LZ, R) of the fused-unpack kernel (last Stockham pass fused into the
# unpack): full traces, partial ones (per-sample loads), odd batches (a CTA
# holding one live trace of two)
VARIANT_CASES = [(5, 1024, 8192), (3, 1000, 8192), (3, 513, 8192),      # LZ 512, R 8
                 (3, 1024, 16384), (2, 777, 16384),                      # LZ 512, R 16
                 (3, 2048, 8192), (3, 1500, 8192),                       # LZ 1024, R 4
                 (4, 2048, 16384), (3, 1025, 16384)]                     # LZ 1024, R 8


@pytest.mark.parametrize("variant", ["fixed", "dual", "fused", "fusedp", "fold", "one"])
def test_fft_kernel_variants_parity(S, monkeypatch, variant):
    # SPEC_FFT_VARIANT pins the kernel variant the autotuner would otherwise
    # choose by timing; every variant must meet the same bar
    monkeypatch.setenv("SPEC_FFT_VARIANT", variant)
    with S.Context(0) as c:
        for batch, n, n_fft in VARIANT_CASES:
            x = traces(batch, n, 7 * n + n_fft)
            got = S.spec_fft(c, dev(x), 20e12, n_fft).cpu().numpy()
            err = rel_rows(got, O.fft_padded(x, n_fft))
            assert err.max() <= TOL, (variant, batch, n, n_fft, err.max())
        # rows at an odd stride (unaligned starts) into a wider output
        for n in (1024, 2048):
            x = traces(3, n, 11 + n)
            base = torch.zeros((3, n + 7), dtype=torch.float32, device="cuda")
            base[:, :n] = dev(x)
            out = torch.full((3, 4200), float("nan"), dtype=torch.complex64, device="cuda")
            S.spec_fft(c, base, 20e12, 8192, n=n, out=out)
            got = out[:, :4097].cpu().numpy()
            assert rel_rows(got, O.fft_padded(x, 8192)).max() <= TOL, (variant, n)
            assert torch.isnan(out[:, 4097:].real).all()


@pytest.mark.parametrize("lanes", ["1", "2"])
def test_zoom_and_bluestein_lane_forms_parity(S, monkeypatch, lanes):
    # SPEC_LANES pins one trace per thread group (1) or two packed traces (2)
    # for the Bluestein and Zoom kernels, which the autotuner otherwise picks
    # by timing; both forms meet the same bar, odd batches included
    monkeypatch.setenv("SPEC_LANES", lanes)
    fs = 20e12
    with S.Context(0) as c:
        for batch, n, f1, f2, d, nt, n_fft in ZOOM_CASES[:9]:
            x = traces(batch, n, 300 + n + d)
            h = O.design_lowpass(nt, d).astype(np.float32)
            got = S.spec_zoom(c, dev(x), fs, f1, f2, d, dev(h), n_fft).cpu().numpy()
            err = rel_rows(got, O.zoom(x, fs, f1, f2, d, h, n_fft))
            assert err.max() <= TOL, (lanes, batch, n, d, nt, n_fft, err.max())
        for batch, n, f1, f2, m in CZT_CASES:
            x = traces(batch, n, 200 + n + m)
            got = S.spec_czt(c, dev(x), fs, f1, f2, m, mode=S.SPEC_CZT_BLUESTEIN).cpu().numpy()
            err = rel_rows(got, O.czt(x, fs, f1, f2, m))
            assert err.max() <= TOL, (lanes, batch, n, m, err.max())


MIXED_CASES = [(4, 500, 2000), (3, 500, 10000), (2, 500, 20000), (3, 1000, 2000), (5, 333, 1050), (3, 12, 42),
               (2, 1, 6), (3, 4000, 26460), (9, 500, 500), (6, 700, 1250)]


@pytest.mark.parametrize("variant", ["mixed", "dftczt"])
def test_fft_non_power_of_two_forms_parity(S, monkeypatch, variant):
    # lengths whose half has only the factors 2, 3, 5, 7: the mixed-radix
    # kernel or the chirp-z on the DFT grid, pinned (the autotuner times both)
    monkeypatch.setenv("SPEC_FFT_VARIANT", variant)
    with S.Context(0) as c:
        for batch, n, n_fft in MIXED_CASES:
            x = traces(batch, n, 5 * n + n_fft)
            got = S.spec_fft(c, dev(x), 20e12, n_fft).cpu().numpy()
            err = rel_rows(got, O.fft_padded(x, n_fft))
            assert err.max() <= TOL, (variant, batch, n, n_fft, err.max())
