"""spec_czt_static -- the chirp-z transform for callers that cannot allocate
device memory (a framework's pool owns it, or a real-time loop must not call
cudaMalloc) -- against the regular spec_czt and the FP64 oracle, called
through the C-ABI.

Calls in a row with different sizes share the library's static working
array; each must match spec_czt (Bluestein) on the same inputs, and the
oracle, within the 1e-5 per-spectrum relative L2 used by every parity test.
The sizes reach every branch of the array's twiddle layout: the largest
N + M - 1 = 8192, a radix plan with a remainder pass (L = 2048, 8192), the
register-only L = 16, and a batch of thousands of traces over many CTAs.  The
file is named to be collected last, and it also passes alone in a fresh
process (the first call does its own per-device set-up)."""
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
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


# (batch, n, f1, f2, m): L = nextpow2(n + m - 1) in the comment
CASES = [(3, 2048, 0.2e12, 2.5e12, 1024),      # L = 4096
         (5, 4096, 0.1e12, 3.6e12, 4097),      # n + m - 1 = 8192 exactly: the array's limit, L = 8192
         (4, 1000, 0.5e12, 1.5e12, 900),       # L = 2048 (16 x 16 x 8: remainder pass)
         (6, 5, 1.0e12, 3.0e12, 8),            # L = 16 (one register-only pass)
         (3000, 1000, 0.8e12, 1.2e12, 512),    # L = 2048, thousands of traces over many CTAs
         (2, 700, 2.0e12, 0.3e12, 300)]        # descending band, L = 1024


def test_static_czt_matches_spec_czt_and_the_oracle_on_calls_in_a_row(S):
    from oracle import spec_oracle as O
    g = np.random.default_rng(2108)
    fs = 20e12
    xs = [g.standard_normal((b, n)).astype(np.float32) for b, n, *_ in CASES]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    # every static call first, back to back, so that consecutive calls change
    # L and the tables in the shared array; then the references
    got = [static_czt(S, x, fs, f1, f2, m) for x, (_, _, f1, f2, m) in zip(xd, CASES)]
    torch.cuda.synchronize()
    got = [X.cpu().numpy() for X in got]
    with S.Context(0) as ctx:
        for x, xh, X, (b, n, f1, f2, m) in zip(xd, xs, got, CASES):
            ref = S.spec_czt(ctx, x, fs, f1, f2, m, mode=S.SPEC_CZT_BLUESTEIN)
            torch.cuda.synchronize()
            err = rel_rows(X, ref.cpu().numpy())
            assert err.max() <= TOL, (b, n, m, err.max())
            pick = np.arange(b) if b <= 8 else np.linspace(0, b - 1, 8).round().astype(np.int64)
            oracle = O.czt(xh[pick], fs, f1, f2, m)
            err_o = rel_rows(X[pick], oracle)
            assert err_o.max() <= TOL, (b, n, m, err_o.max())


def test_static_czt_second_call_after_a_larger_one_is_unaffected(S):
    # the largest tables first, then a small call: nothing left over in the
    # shared array may leak into the smaller transform
    from oracle import spec_oracle as O
    g = np.random.default_rng(7)
    fs = 20e12
    big = torch.from_numpy(g.standard_normal((2, 4096)).astype(np.float32)).cuda()
    small_h = g.standard_normal((3, 40)).astype(np.float32)
    small = torch.from_numpy(small_h).cuda()
    for _ in range(2):
        static_czt(S, big, fs, 0.1e12, 3.6e12, 4097)
        X = static_czt(S, small, fs, 0.3e12, 0.9e12, 25)
        torch.cuda.synchronize()
        err = rel_rows(X.cpu().numpy(), O.czt(small_h, fs, 0.3e12, 0.9e12, 25))
        assert err.max() <= TOL, err


def test_static_czt_rejects_sizes_beyond_its_array(S):
    x = torch.zeros((1, 6000), device="cuda")
    X = torch.zeros((1, 4000), dtype=torch.complex64, device="cuda")
    st = S.lib().spec_czt_static(x.data_ptr(), 1, 6000, 6000, 1.0, 0.1, 0.2, 4000, X.data_ptr(), 4000, None)
    assert st == S.SPEC_EUNSUPPORTED
    # one past the limit: n + m - 1 = 8193
    X2 = torch.zeros((1, 4097), dtype=torch.complex64, device="cuda")
    st = S.lib().spec_czt_static(x.data_ptr(), 1, 4097, 6000, 1.0, 0.1, 0.2, 4097, X2.data_ptr(), 4097, None)
    assert st == S.SPEC_EUNSUPPORTED
    # sizes near 2^62 are rejected before n + m - 1 is formed
    st = S.lib().spec_czt_static(x.data_ptr(), 1, 1 << 62, 1 << 62, 1.0, 0.1, 0.2, 1 << 62, X.data_ptr(),
                                 1 << 62, None)
    assert st == S.SPEC_EUNSUPPORTED
    # host buffers would need staging memory
    xh = np.zeros((1, 64), np.float32)
    Xh = np.zeros((1, 8), np.complex64)
    st = S.lib().spec_czt_static(xh.ctypes.data, 1, 64, 64, 1.0, 0.1, 0.2, 8, Xh.ctypes.data, 8, None)
    assert st == S.SPEC_EINVAL
