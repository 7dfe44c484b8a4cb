"""spec_czt_static -- the chirp-z transform for callers that cannot allocate
device memory (a framework's pool owns it, or a real-time loop must not call
cudaMalloc) -- against the regular spec_czt, called through the C-ABI.

Two calls in a row with different sizes share the library's static working
array; each must match spec_czt on the same inputs within the 1e-5
per-spectrum relative L2 used by every parity test.  The file is named to be
collected last, and it also passes alone in a fresh process (the first call
does its own per-device set-up)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def S():
    from paper_2108_03948_gb300 import build
    build.build()
    from paper_2108_03948_gb300 import spec
    spec.lib()
    return spec


def static_czt(S, x, fs, f1, f2, m):
    X = torch.full((x.shape[0], m), float("nan"), dtype=torch.complex64, device="cuda")
    st = S.lib().spec_czt_static(x.data_ptr(), x.shape[0], x.shape[1], x.stride(0), fs, f1, f2, m,
                                 X.data_ptr(), X.stride(0), torch.cuda.current_stream().cuda_stream)
    assert st == S.SPEC_OK
    return X


def rel_rows(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def test_static_czt_matches_spec_czt_on_two_calls_in_a_row(S):
    g = np.random.default_rng(2108)
    fs = 20e12
    cases = [(3, 2048, 0.2e12, 2.5e12, 1024),      # L = 4096
             (5, 1000, 0.1e12, 3.6e12, 2047)]      # L = 4096, other tables
    xs = [torch.from_numpy(g.standard_normal((b, n)).astype(np.float32)).cuda() for b, n, *_ in cases]
    got = [static_czt(S, x, fs, f1, f2, m) for x, (_, _, f1, f2, m) in zip(xs, cases)]
    torch.cuda.synchronize()
    with S.Context(0) as ctx:
        for x, X, (_, _, f1, f2, m) in zip(xs, got, cases):
            ref = S.spec_czt(ctx, x, fs, f1, f2, m, mode=S.SPEC_CZT_BLUESTEIN)
            torch.cuda.synchronize()
            err = rel_rows(X, ref)
            assert err.max() <= TOL, err


def test_static_czt_rejects_sizes_beyond_its_array(S):
    x = torch.zeros((1, 6000), device="cuda")
    X = torch.zeros((1, 4000), dtype=torch.complex64, device="cuda")
    st = S.lib().spec_czt_static(x.data_ptr(), 1, 6000, 6000, 1.0, 0.1, 0.2, 4000, X.data_ptr(), 4000, None)
    assert st == S.SPEC_EUNSUPPORTED
    # host buffers would need staging memory
    xh = np.zeros((1, 64), np.float32)
    Xh = np.zeros((1, 8), np.complex64)
    st = S.lib().spec_czt_static(xh.ctypes.data, 1, 64, 64, 1.0, 0.1, 0.2, 8, Xh.ctypes.data, 8, None)
    assert st == S.SPEC_EINVAL
