"""Long traces: the multi-pass FFT and Bluestein paths, the segmented chirp-z
(N >> M) and the large Zoom path against the FP64 oracle.  Where the oracle can afford every bin the
comparison is element by element over the whole spectrum; at the largest
sizes (262144-sample traces, N_FFT up to 2^24) it is over a fixed sample of
bins -- both band edges, the ends of the range and a seeded spread -- each
computed by its own direct sum.  The bar is relative L2 <= 1e-5 per
spectrum (over the sample where sampled)."""
import numpy as np
import pytest

from oracle import spec_oracle as O
from paper_2108_03948_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
FS = synth.FS


@pytest.fixture(scope="module")
def S():
    from paper_2108_03948_gb300 import build
    build.build()
    from paper_2108_03948_gb300 import spec
    return spec


@pytest.fixture(scope="module")
def ctx(S):
    c = S.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    return np.linalg.norm(got - ref, axis=-1) / np.linalg.norm(ref, axis=-1)


def sample(total, count, seed):
    g = np.random.default_rng(seed)
    ends = [0, 1, 2, total // 2 - 1, total // 2, total // 2 + 1, total - 2, total - 1]
    return np.unique(np.concatenate([ends, g.integers(0, total, count)]).clip(0, total - 1))


def noise(batch, n, seed):
    return np.random.default_rng(seed).standard_normal((batch, n)).astype(np.float32)


# ------------------------------------------------------------------- FFT ---

@pytest.mark.parametrize("batch,n,n_fft", [(2, 20000, 32768), (3, 100, 262144), (2, 16385, 32768)])
def test_long_fft_full(ctx, S, batch, n, n_fft):
    x = noise(batch, n, n)
    got = S.spec_fft(ctx, dev(x), FS, n_fft).cpu().numpy()
    assert rel(got, O.fft_padded(x, n_fft)).max() <= TOL


@pytest.mark.parametrize("batch,n,n_fft,kind", [(3, 262144, 1 << 21, "thz"), (2, 262143, 1 << 19, "noise"),
                                                (1, 3_000_000, 1 << 24, "noise")])
def test_long_fft_sampled(ctx, S, batch, n, n_fft, kind):
    x = synth.batch_traces(4, range(batch), n=n) if kind == "thz" else noise(batch, n, 7)
    got = S.spec_fft(ctx, dev(x), FS, n_fft).cpu().numpy()
    assert got.shape == (batch, n_fft // 2 + 1)
    k = sample(n_fft // 2 + 1, 120 if n > 1_000_000 else 250, n)
    assert rel(got[:, k], O.fft_padded_bins(x, n_fft, k)).max() <= TOL
    assert np.isfinite(got).all()


# ------------------------------------------------------------------- CZT ---

@pytest.mark.parametrize("batch,n,f1,f2,m", [
    # multi-pass Bluestein (M > 8192)
    (2, 12000, 0.2e12, 2.5e12, 9000),      # L = 32768, two residues in the column pass
    (2, 1000, 0.1e12, 5.0e12, 40000),      # M > N
    (2, 30000, 0.3e12, 0.6e12, 8193),      # just above the segmented limit
    (2, 5000, 3.0e12, 0.5e12, 20000),      # f2 < f1 (negative step)
    # segmented (N + M - 1 > 16384, M <= 8192)
    (2, 12000, 0.2e12, 2.5e12, 8000),      # two segments of a 16384-point Bluestein
    (2, 30000, 0.3e12, 0.31e12, 100),      # 8192-point segments, ragged last segment
    (2, 20000, 1.0e12, 1.0e12, 1),         # M = 1
    (2, 17000, 3.0e12, 0.5e12, 3000),      # f2 < f1 (negative step)
    (3, 16385, 0.1e12, 9.9e12, 1),         # one sample past the one-CTA limit
    (2, 3 * 6145, 0.5e12, 1.5e12, 2048),   # exactly three 8192-point segments
    (2, 40000, 0.5e12, 1.5e12, 2049),      # 16384-point segments from M = 2049
])
def test_long_czt_full(ctx, S, batch, n, f1, f2, m):
    x = noise(batch, n, m)
    got = S.spec_czt(ctx, dev(x), FS, f1, f2, m).cpu().numpy()
    assert got.shape == (batch, m)
    assert rel(got, O.czt(x, FS, f1, f2, m)).max() <= TOL


def test_long_czt_workload4_sampled(ctx, S):
    cfg = synth.UNIFORM[4]
    x = synth.batch_traces(4, range(3))
    got = S.spec_czt(ctx, dev(x), cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m).cpu().numpy()
    k = sample(cfg.czt_m, 250, 4)
    ref = O.czt_bins(x, cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m, k)
    assert rel(got[:, k], ref).max() <= TOL
    assert np.isfinite(got).all()


def test_segmented_czt_narrow_band_of_long_traces(ctx, S):
    # the THz use case of N >> M: a 1024-point 0.3-0.4 THz band of
    # 262144-sample traces, 33 segments of an 8192-point Bluestein
    cfg = synth.UNIFORM[4]
    x = synth.batch_traces(4, range(3))
    got = S.spec_czt(ctx, dev(x), cfg.fs, 0.3e12, 0.4e12, 1024).cpu().numpy()
    k = sample(1024, 250, 6)
    assert rel(got[:, k], O.czt_bins(x, cfg.fs, 0.3e12, 0.4e12, 1024, k)).max() <= TOL


def test_long_czt_table_cache_and_repeat(ctx, S):
    # the second call reuses the cached multi-pass tables and gives the same bits
    x = dev(noise(2, 15000, 3))
    a = S.spec_czt(ctx, x, FS, 0.5e12, 1.5e12, 4000)
    b = S.spec_czt(ctx, x, FS, 0.5e12, 1.5e12, 4000)
    assert torch.equal(torch.view_as_real(a), torch.view_as_real(b))


# ------------------------------------------------------------------ Zoom ---

def test_zoom_workload4_sampled(ctx, S):
    cfg = synth.UNIFORM[4]
    x = synth.batch_traces(4, range(2))
    h = O.design_lowpass(cfg.zoom_taps, cfg.zoom_d).astype(np.float32)
    got = S.spec_zoom(ctx, dev(x), cfg.fs, cfg.zoom_f1, cfg.zoom_f2, cfg.zoom_d, dev(h),
                      cfg.zoom_n_fft).cpu().numpy()
    K = cfg.zoom_n_fft // cfg.zoom_d
    k = sample(K, 250, 5)
    ref = O.zoom_bins(x, cfg.fs, cfg.zoom_f1, cfg.zoom_f2, cfg.zoom_d, h, cfg.zoom_n_fft, k)
    assert rel(got[:, k], ref).max() <= TOL


# ------------------------------------------------------ host buffers ------

def test_long_paths_host_pipeline_chunks(ctx, S):
    """Host buffers above 16 MiB of traffic run in chunks of traces: the
    multi-pass FFT (20 traces to 2^18) and the segmented chirp-z (21 traces of
    262144 samples, a 1024-bin band) give the device-pointer call's bits."""
    x = noise(20, 200000, 12)
    Xd = S.spec_fft(ctx, dev(x), FS, 1 << 18).cpu().numpy()
    Xh = S.spec_fft(ctx, x, FS, 1 << 18)
    assert np.array_equal(np.asarray(Xh), Xd)
    y = noise(21, 262144, 13)
    Zd = S.spec_czt(ctx, dev(y), FS, 0.3e12, 0.4e12, 1024).cpu().numpy()
    Zh = S.spec_czt(ctx, y, FS, 0.3e12, 0.4e12, 1024)
    assert np.array_equal(np.asarray(Zh), Zd)


def test_long_paths_with_host_buffers(ctx, S):
    x = noise(2, 40000, 11)
    Xd = S.spec_fft(ctx, dev(x), FS, 65536).cpu().numpy()
    Xh = S.spec_fft(ctx, x, FS, 65536)
    assert np.array_equal(np.asarray(Xh), Xd)
    Zd = S.spec_czt(ctx, dev(x), FS, 0.2e12, 1.2e12, 3000).cpu().numpy()
    Zh = S.spec_czt(ctx, x, FS, 0.2e12, 1.2e12, 3000)
    assert np.array_equal(np.asarray(Zh), Zd)
