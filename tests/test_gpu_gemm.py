"""Chirp-z as a tensor-core product (SPEC_CZT_GEMM_F16X3 / _F16X1): parity
with the FP64 oracle element by element, on shapes that leave ragged tiles
in every dimension (traces not a multiple of 128, samples not a multiple of
64, 2M not a multiple of 128), the degenerate M = 1 and descending bands,
the full workload-3 batch in the bench's launch configuration (sampled
traces), and the bounded-wait machinery."""
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


def noise(batch, n, seed):
    return np.random.default_rng(seed).standard_normal((batch, n)).astype(np.float32)


CASES = [
    (300, 1024, 0.8e12, 1.2e12, 512),      # workload-3 shape
    (129, 1000, 0.2e12, 2.5e12, 100),      # ragged in every dimension
    (5, 37, 0.1e12, 9.0e12, 3),
    (3, 2048, 0.2e12, 2.5e12, 1024),       # workload-1 shape
    (4, 500, 1.3e12, 1.3e12, 1),           # M = 1
    (7, 777, 3.0e12, 0.4e12, 257),         # descending band
    (2, 4096, 0.0, 10.0e12, 2048),
]


@pytest.mark.parametrize("batch,n,f1,f2,m", CASES)
def test_gemm_f16x3_parity(ctx, S, batch, n, f1, f2, m):
    x = noise(batch, n, n + m)
    got = S.spec_czt(ctx, dev(x), FS, f1, f2, m, mode=S.SPEC_CZT_GEMM_F16X3).cpu().numpy()
    assert got.shape == (batch, m)
    assert rel(got, O.czt(x, FS, f1, f2, m)).max() <= TOL


def test_gemm_f16x3_scale_invariance(ctx, S):
    # per-row power-of-two scaling: rows of very different magnitude
    x = noise(6, 1024, 1)
    x *= np.array([1e-30, 1e-8, 1.0, 3e5, 1e20, 1e30], dtype=np.float32)[:, None]
    got = S.spec_czt(ctx, dev(x), FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_GEMM_F16X3).cpu().numpy()
    assert rel(got, O.czt(x, FS, 0.8e12, 1.2e12, 512)).max() <= TOL


def test_gemm_thz_traces(ctx, S):
    cfg = synth.UNIFORM[3]
    x = synth.batch_traces(3, range(200))
    got = S.spec_czt(ctx, dev(x), cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m, mode=S.SPEC_CZT_GEMM_F16X3)
    ref = O.czt(x, cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m)
    assert rel(got.cpu().numpy(), ref).max() <= TOL


def test_gemm_f16x1_is_the_low_precision_form(ctx, S):
    x = noise(64, 1024, 2)
    got = S.spec_czt(ctx, dev(x), FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_GEMM_F16X1).cpu().numpy()
    err = rel(got, O.czt(x, FS, 0.8e12, 1.2e12, 512))
    assert err.max() <= 3e-3
    assert err.max() > 1e-6           # it really is the one-product form


def test_gemm_bf16x1_is_the_single_term_bf16_error(ctx, S):
    # x and Z rounded once to BF16 (8-bit significands, unit roundoff 2^-9),
    # one product accumulated in FP32: relative error of order 1e-3 per
    # spectrum, several times the FP16 one-product form's (11-bit significands)
    x = noise(64, 1024, 2)
    ref = O.czt(x, FS, 0.8e12, 1.2e12, 512)
    got = S.spec_czt(ctx, dev(x), FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_GEMM_BF16X1).cpu().numpy()
    f16 = S.spec_czt(ctx, dev(x), FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_GEMM_F16X1).cpu().numpy()
    err, err16 = rel(got, ref), rel(f16, ref)
    assert 3e-4 < err.max() <= 2e-2
    assert err.mean() > 3 * err16.mean()
    # the FP16 split form stays at the FP32 level on the same traces
    split = S.spec_czt(ctx, dev(x), FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_GEMM_F16X3).cpu().numpy()
    assert rel(split, ref).max() <= 1e-5


def test_gemm_matches_bluestein(ctx, S):
    x = dev(noise(256, 1024, 3))
    g = S.spec_czt(ctx, x, FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_GEMM_F16X3).cpu().numpy()
    b = S.spec_czt(ctx, x, FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_BLUESTEIN).cpu().numpy()
    assert rel(g, b.astype(np.complex128)).max() <= 2e-6


def test_gemm_host_buffers_and_repeat(ctx, S):
    x = noise(130, 700, 4)
    d = S.spec_czt(ctx, dev(x), FS, 0.5e12, 1.5e12, 300, mode=S.SPEC_CZT_GEMM_F16X3).cpu().numpy()
    d2 = S.spec_czt(ctx, dev(x), FS, 0.5e12, 1.5e12, 300, mode=S.SPEC_CZT_GEMM_F16X3).cpu().numpy()
    h = S.spec_czt(ctx, x, FS, 0.5e12, 1.5e12, 300, mode=S.SPEC_CZT_GEMM_F16X3)
    assert np.array_equal(d, d2)
    assert np.array_equal(np.asarray(h), d)


def test_gemm_and_spiral_host_pipeline_chunks(ctx, S):
    """Host buffers above 16 MiB run in overlapped chunks of traces; each row
    of the product is computed by the same MMA sequence wherever its tile
    lies, so the chunked host call equals the device-pointer call bit for
    bit (4000 traces: chunks of 1024 and a ragged last one), on the unit
    circle and off it."""
    x = noise(4000, 1024, 9)
    xd = dev(x)
    d = S.spec_czt(ctx, xd, FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_GEMM_F16X3).cpu().numpy()
    h = S.spec_czt(ctx, x, FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_GEMM_F16X3)
    assert np.array_equal(np.asarray(h), d)
    ds = S.spec_czt_spiral(ctx, xd, FS, 0.8e12, 1.2e12, 512, 1.0005, 0.9999).cpu().numpy()
    hs = np.zeros((4000, 515), dtype=np.complex64)
    S.spec_czt_spiral(ctx, x, FS, 0.8e12, 1.2e12, 512, 1.0005, 0.9999, out=hs[:, :512])
    assert np.array_equal(hs[:, :512], ds)
    assert not hs[:, 512:].any()
    torch.cuda.synchronize()
    assert S.ctx_status(ctx) == S.SPEC_OK


def test_workload3_full_batch_sampled(ctx, S):
    cfg = synth.UNIFORM[3]
    idx = np.arange(cfg.batch)
    x = synth.batch_traces(3, range(1024))
    xall = np.tile(x, (cfg.batch // 1024, 1))         # 65536 traces, 64 copies of 1024 distinct ones
    got = S.spec_czt(ctx, dev(xall), cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m, mode=S.SPEC_CZT_GEMM_F16X3)
    torch.cuda.synchronize()
    assert S.ctx_status(ctx) == S.SPEC_OK
    g = got.cpu().numpy()
    assert np.isfinite(g).all()
    pick = [0, 1, 127, 128, 1023]
    ref = O.czt(x[pick], cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m)
    for r in (0, 5, 63):                             # the same traces in different tiles give the same bits
        assert rel(g[r * 1024 + np.array(pick)], ref).max() <= TOL
    assert np.array_equal(g[idx[:1024]], g[idx[-1024:]])


def test_bounded_wait_reports_timeout_and_context_survives(ctx, S):
    assert S.ctx_status(ctx) == S.SPEC_OK
    S.spec_selftest_wait_timeout(ctx, 2000)                 # a 2 ms wait on a barrier nothing completes
    assert S.ctx_status(ctx) == S.SPEC_ETIMEOUT
    assert S.ctx_status(ctx) == S.SPEC_OK                   # reading clears it
    x = noise(2, 256, 9)
    got = S.spec_czt(ctx, dev(x), FS, 0.5e12, 1.0e12, 64, mode=S.SPEC_CZT_GEMM_F16X3).cpu().numpy()
    assert rel(got, O.czt(x, FS, 0.5e12, 1.0e12, 64)).max() <= TOL


def test_auto_mode_is_measured_and_equals_the_chosen_mode(ctx, S):
    # AUTO's choice comes from timing both exact forms on a probe batch; the
    # spectra of an AUTO call equal those of the explicit chosen mode bit for
    # bit.  At the workload-3 shape (65536 x 1024, M = 512) the product wins;
    # at the workload-1 shape (4096 x 2048, M = 1024, L = 4096) Bluestein does.
    x3 = dev(np.tile(noise(1024, 1024, 5), (64, 1)))
    m3 = S.spec_czt_auto_mode(ctx, x3.shape[0], 1024, FS, 0.8e12, 1.2e12, 512)
    a = S.spec_czt(ctx, x3, FS, 0.8e12, 1.2e12, 512)
    g = S.spec_czt(ctx, x3, FS, 0.8e12, 1.2e12, 512, mode=m3)
    assert torch.equal(torch.view_as_real(a), torch.view_as_real(g))
    assert m3 == S.SPEC_CZT_GEMM_F16X3
    x1 = dev(noise(4096, 2048, 6))
    m1 = S.spec_czt_auto_mode(ctx, 4096, 2048, FS, 0.2e12, 2.5e12, 1024)
    a = S.spec_czt(ctx, x1, FS, 0.2e12, 2.5e12, 1024)
    b = S.spec_czt(ctx, x1, FS, 0.2e12, 2.5e12, 1024, mode=m1)
    assert torch.equal(torch.view_as_real(a), torch.view_as_real(b))
    assert m1 == S.SPEC_CZT_BLUESTEIN


def test_auto_mode_decisions_persist_to_the_cache_file(S, tmp_path, monkeypatch):
    import json
    path = tmp_path / "tune.json"
    monkeypatch.setenv("SPEC_AUTOTUNE_CACHE", str(path))
    with S.Context(0) as c:
        mode = S.spec_czt_auto_mode(c, 8192, 1024, FS, 0.8e12, 1.2e12, 512)
    d = json.loads(path.read_text())
    assert d["format"] == "spec-autotune-1"
    key = "czt n=1024 m=512 b=8192"
    value = d["entries"][key]            # beside it: the kernel-variant choices the probe runs made
    assert value == ("gemm_f16x3" if mode == S.SPEC_CZT_GEMM_F16X3 else "bluestein")
    # a new context reads the decision instead of measuring; a planted value
    # shows that the file, not a new measurement, decided
    planted = "bluestein" if value == "gemm_f16x3" else "gemm_f16x3"
    assert S.spec_tune_cache_store(str(path), d["device"], key, planted) == 0
    with S.Context(0) as c:
        again = S.spec_czt_auto_mode(c, 8192, 1024, FS, 0.8e12, 1.2e12, 512)
    assert again == (S.SPEC_CZT_GEMM_F16X3 if planted == "gemm_f16x3" else S.SPEC_CZT_BLUESTEIN)


def test_gemm_large_batch_matches_small_calls(ctx, S):
    # many tiles per CTA of the persistent grid: every copy of a trace gives
    # the same bits as a call with that trace block alone
    x = noise(1024, 1024, 8)
    xall = dev(np.tile(x, (48, 1)))                          # 49152 traces: 3 chunks
    big = S.spec_czt(ctx, xall, FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_GEMM_F16X3)
    one = S.spec_czt(ctx, dev(x), FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_GEMM_F16X3)
    torch.cuda.synchronize()
    b = big.view(48, 1024, 512)
    for r in (0, 17, 33, 47):
        assert torch.equal(torch.view_as_real(b[r]), torch.view_as_real(one))


# ------------------------------------------------------ off the unit circle

SPIRALS = [
    (4, 1024, 0.8e12, 1.2e12, 512, 0.999, 1.0001),
    (3, 1000, 0.2e12, 2.5e12, 300, 1.01, 0.9999),
    (5, 500, 0.1e12, 5.0e12, 100, 0.98, 1.001),        # column scales up to ~2^86
    (129, 77, 3.0e12, 0.5e12, 33, 1.002, 0.998),       # descending band, ragged tiles
]


@pytest.mark.parametrize("batch,n,f1,f2,m,a0,w0", SPIRALS)
def test_spiral_czt_parity(ctx, S, batch, n, f1, f2, m, a0, w0):
    x = noise(batch, n, n + m + 1)
    got = S.spec_czt_spiral(ctx, dev(x), FS, f1, f2, m, a0, w0).cpu().numpy()
    assert rel(got, O.czt_spiral(x, FS, f1, f2, m, a0, w0)).max() <= TOL


def test_spiral_czt_on_the_unit_circle_is_the_gemm_czt(ctx, S):
    x = dev(noise(300, 1024, 21))
    a = S.spec_czt_spiral(ctx, x, FS, 0.8e12, 1.2e12, 512, 1.0, 1.0)
    b = S.spec_czt(ctx, x, FS, 0.8e12, 1.2e12, 512, mode=S.SPEC_CZT_GEMM_F16X3)
    assert torch.equal(torch.view_as_real(a), torch.view_as_real(b))


def test_spiral_czt_rejections(ctx, S):
    lib = S.lib()
    x = torch.zeros((2, 1000), device="cuda")
    X = torch.zeros((2, 64), dtype=torch.complex64, device="cuda")
    args = (ctx.handle, x.data_ptr(), 2, 1000, 1000, FS, 0.1e12, 1.0e12, 64)
    assert lib.spec_czt_spiral(*args, 0.0, 1.0, X.data_ptr(), 64, None) == S.SPEC_EINVAL
    assert lib.spec_czt_spiral(*args, 1.0, -1.0, X.data_ptr(), 64, None) == S.SPEC_EINVAL
    assert lib.spec_czt_spiral(*args, 0.5, 1.0, X.data_ptr(), 64, None) == S.SPEC_EUNSUPPORTED   # 2^999
    assert np.all(X.cpu().numpy() == 0)


@pytest.mark.parametrize("batch,m,ld", [(300, 512, 600), (129, 100, 104), (131, 48, 48)])
def test_gemm_output_pitch_and_edges(ctx, S, batch, m, ld):
    # the product's epilogue stores 32 x 32 boxes with bulk tensor copies when
    # the output rows are 16-byte aligned: a row pitch wider than M, a batch
    # that ends inside a 128-row tile and 2M not a multiple of 32 must all
    # leave every byte outside the spectra untouched
    x = noise(batch, 1000, batch + m)
    out = torch.full((batch, ld), complex(float("nan"), float("nan")), dtype=torch.complex64, device="cuda")
    S.spec_czt(ctx, dev(x), FS, 0.3e12, 2.2e12, m, mode=S.SPEC_CZT_GEMM_F16X3, out=out)
    got = out.cpu().numpy()
    assert rel(got[:, :m], O.czt(x, FS, 0.3e12, 2.2e12, m)).max() <= TOL
    if ld > m:
        assert np.isnan(got[:, m:].real).all() and np.isnan(got[:, m:].imag).all()


def test_gemm_with_the_split_inside_the_product(S, monkeypatch):
    # SPEC_GEMM_FUSED=1: x is read as FP32 boxes by TMA and split into the FP16
    # parts by converter warps inside the product; the parts are the same bits
    # as the separate split pass's, so the spectra are identical
    x = dev(noise(300, 1000, 77))
    with S.Context(0) as c0:
        ref = S.spec_czt(c0, x, FS, 0.3e12, 2.2e12, 256, mode=S.SPEC_CZT_GEMM_F16X3)
        ref1 = S.spec_czt(c0, x, FS, 0.3e12, 2.2e12, 256, mode=S.SPEC_CZT_GEMM_BF16X1)
    monkeypatch.setenv("SPEC_GEMM_FUSED", "1")
    with S.Context(0) as c1:
        got = S.spec_czt(c1, x, FS, 0.3e12, 2.2e12, 256, mode=S.SPEC_CZT_GEMM_F16X3)
        got1 = S.spec_czt(c1, x, FS, 0.3e12, 2.2e12, 256, mode=S.SPEC_CZT_GEMM_BF16X1)
    assert torch.equal(torch.view_as_real(got), torch.view_as_real(ref))
    assert torch.equal(torch.view_as_real(got1), torch.view_as_real(ref1))
    assert rel(got.cpu().numpy(), O.czt(x.cpu().numpy(), FS, 0.3e12, 2.2e12, 256)).max() <= TOL
