"""Ragged batches (spec_ragged): traces with their own length, band, point
count, decimation and taps in one call.  Every trace must match the same
trace run alone through spec_fft / spec_czt / spec_zoom to 2e-6 relative L2
(the plan's autotuner may pick a different kernel variant -- lanes, pass
radix, cluster -- and the ragged chirp-z evaluates its chirps in the kernel,
so the rounding differs in the last bits), and every trace is checked
against the FP64 oracle (relative L2 <= 1e-5 per spectrum).  The plan's CUDA graph replay is bit-identical to its first
run, and the graph is re-captured when the pools move."""
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


def workload(count, seed=5):
    """Workload-2-shaped traces and parameters, with some extremes mixed in."""
    rg = synth.ragged_params(count)
    items = list(rg.items)
    items[0] = synth.RaggedTrace(8192, 65536, 0.1e12, 3.9e12, 4096, 2, 127)    # largest of each
    items[1] = synth.RaggedTrace(1000, 8192, 0.1e12, 0.6e12, 256, 16, 31)      # smallest
    traces = [synth.ragged_trace(i, it) for i, it in enumerate(items)]
    return items, traces


def pools(items, traces, kind):
    xo, x_all = [], []
    off = 0
    for t in traces:
        xo.append(off)
        x_all.append(t)
        off += len(t) + 3                              # gaps between traces
        x_all.append(np.zeros(3, np.float32))
    x_pool = torch.from_numpy(np.concatenate(x_all)).cuda()
    bins = []
    for it in items:
        bins.append(it.n_fft // 2 + 1 if kind == 0 else it.m if kind == 1 else it.n_fft // it.d)
    oo = np.concatenate([[0], np.cumsum(bins)[:-1]]).astype(np.int64)
    X_pool = torch.full((int(np.sum(bins)),), float("nan"), dtype=torch.complex64, device="cuda")
    taps, to = [], []
    toff = 0
    for it in items:
        h = O.design_lowpass(it.n_taps, it.d).astype(np.float32)
        taps.append(h)
        to.append(toff)
        toff += len(h)
    taps_pool = torch.from_numpy(np.concatenate(taps)).cuda()
    descs = [dict(x_off=int(xo[i]), n=it.n, out_off=int(oo[i]), f1=it.f1, f2=it.f2, n_fft=it.n_fft, m=it.m,
                  d=it.d, taps_off=int(to[i]), n_taps=it.n_taps) for i, it in enumerate(items)]
    return descs, x_pool, X_pool, taps_pool, bins, taps


def single(S, ctx, kind, it, x, h):
    xd = torch.from_numpy(x[None, :]).cuda()
    if kind == 0:
        return S.spec_fft(ctx, xd, FS, it.n_fft)[0]
    if kind == 1:
        return S.spec_czt(ctx, xd, FS, it.f1, it.f2, it.m)[0]
    return S.spec_zoom(ctx, xd, FS, it.f1, it.f2, it.d, torch.from_numpy(h).cuda(), it.n_fft)[0]


_ORACLE = {}


def oracle(kind, it, x, h):
    """The FP64 oracle's spectrum, computed once per (kind, trace) and reused
    by the tests that check both forms of a plan."""
    key = (kind, it.n, it.n_fft, it.f1, it.f2, it.m, it.d, it.n_taps, x.tobytes(), np.asarray(h).tobytes())
    if key not in _ORACLE:
        _ORACLE[key] = _oracle(kind, it, x, h)
    return _ORACLE[key]


def _oracle(kind, it, x, h):
    if kind == 0:
        return O.fft_padded(x, it.n_fft)[0]
    if kind == 1:
        return O.czt(x, FS, it.f1, it.f2, it.m)[0]
    return O.zoom(x, FS, it.f1, it.f2, it.d, h, it.n_fft)[0]


@pytest.fixture(scope="module")
def forced(S):
    """Contexts whose ragged plans always (1) or never (0) use the work
    queue (SPEC_RAGGED_QUEUE is read when a context is created)."""
    import os
    out = {}
    for v in (1, 0):
        os.environ["SPEC_RAGGED_QUEUE"] = str(v)
        out[v] = S.Context(0)
    del os.environ["SPEC_RAGGED_QUEUE"]
    yield out
    for c in out.values():
        c.close()


@pytest.mark.parametrize("form", ["queue", "classes"])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_ragged_matches_single_calls_and_oracle(S, ctx, forced, kind, form):
    # both forms a plan can take: the persistent work queue and the per-shape
    # launches, each against single calls and (every trace) the oracle
    rc = forced[1 if form == "queue" else 0]
    items, traces = workload(48)
    descs, x_pool, X_pool, taps_pool, bins, taps = pools(items, traces, kind)
    S.spec_ragged(rc, kind, descs, FS, x_pool, X_pool, taps_pool)
    assert S.spec_ragged_plan_info(rc, kind, descs, FS)[0] == (form == "queue")
    first = X_pool.clone()
    S.spec_ragged(rc, kind, descs, FS, x_pool, X_pool, taps_pool)       # graph replay
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(first), torch.view_as_real(X_pool))
    got = X_pool.cpu().numpy()
    for i, it in enumerate(items):
        o, nb = descs[i]["out_off"], bins[i]
        ref = single(S, ctx, kind, it, traces[i], taps[i]).cpu().numpy()
        d = np.linalg.norm(got[o:o + nb] - ref) / np.linalg.norm(ref)
        assert d <= 2e-6, (i, d)
        r = oracle(kind, it, traces[i], taps[i])
        err = np.linalg.norm(got[o:o + nb] - r) / np.linalg.norm(r)
        assert err <= TOL, (i, err)


def test_ragged_recaptures_when_pools_move(S, ctx):
    items, traces = workload(12)
    descs, x_pool, X_pool, taps_pool, bins, taps = pools(items, traces, 1)
    S.spec_ragged(ctx, 1, descs, FS, x_pool, X_pool, taps_pool)
    x2 = x_pool.clone()
    X2 = torch.zeros_like(X_pool)
    S.spec_ragged(ctx, 1, descs, FS, x2, X2, taps_pool)
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(X_pool), torch.view_as_real(X2))


def test_ragged_rejects_bad_descriptors(S, ctx):
    lib = S.lib()
    x = torch.zeros(64, device="cuda")
    X = torch.zeros(64, dtype=torch.complex64, device="cuda")
    bad = (S.spec_desc * 2)(S.spec_desc(0, 64, 0, 0, 0, 64, 0, 0, 0, 0), S.spec_desc(0, 64, 0, 0, 0, 48, 0, 0, 0, 0))
    st = lib.spec_ragged(ctx.handle, 0, bad, 2, FS, x.data_ptr(), None, X.data_ptr(), None)
    assert st == S.SPEC_EINVAL
    assert b"descriptor 1" in lib.spec_last_error(ctx.handle)
    # host pools are refused
    xh = np.zeros(64, np.float32)
    st = lib.spec_ragged(ctx.handle, 0, bad, 1, FS, xh.ctypes.data, None, X.data_ptr(), None)
    assert st == S.SPEC_EINVAL


def test_ragged_czt_odd_class_with_two_traces_per_cta(S, ctx):
    # L = 2048 runs two traces per CTA; an odd count leaves a dead slot in the
    # last CTA, which must read only valid tables and write nothing.
    items = [synth.RaggedTrace(1000, 8192, 0.2e12 + 0.1e12 * i, 1.5e12, 300 + 7 * i, 2, 31) for i in range(3)]
    traces = [synth.ragged_trace(i, it) for i, it in enumerate(items)]
    descs, x_pool, X_pool, taps_pool, bins, taps = pools(items, traces, 1)
    S.spec_ragged(ctx, 1, descs, FS, x_pool, X_pool, taps_pool)
    torch.cuda.synchronize()
    got = X_pool.cpu().numpy()
    for i, it in enumerate(items):
        o, nb = descs[i]["out_off"], bins[i]
        r = oracle(1, it, traces[i], taps[i])
        assert np.linalg.norm(got[o:o + nb] - r) / np.linalg.norm(r) <= TOL


def test_ragged_czt_queue_units_and_shared_kernel_spectra(S, forced):
    ctx = forced[1]
    # The chirp-z work queue packs 8192/L traces per unit: 1030 traces of
    # L = 16 make three units (the last with dead slots), mixed with longer
    # classes; repeated (N, M, band) share one FFT(v)/L table.  Every trace
    # must match the oracle, and the repeats must equal their originals.
    rng = np.random.default_rng(11)
    items = []
    for i in range(1030):
        items.append(synth.RaggedTrace(5, 64, 0.1e12 + 1e9 * (i % 7), 3.0e12, 8, 2, 31))
    for i in range(9):
        n = int(rng.integers(1000, 8193))
        items.append(synth.RaggedTrace(n, 65536, 0.3e12, 0.3e12 + 0.1e12 * (i + 1), int(rng.integers(256, 4097)),
                                       2, 31))
    items.append(items[-1])
    # standard-normal samples: 5-sample THz traces would be all zero
    traces = [rng.standard_normal(it.n).astype(np.float32) for it in items]
    traces[-1] = traces[-2]
    descs, x_pool, X_pool, taps_pool, bins, taps = pools(items, traces, 1)
    S.spec_ragged(ctx, 1, descs, FS, x_pool, X_pool, taps_pool)
    torch.cuda.synchronize()
    got = X_pool.cpu().numpy()
    assert S.spec_ragged_launches(ctx, 1, descs, FS) == 1
    for i in list(range(0, 1030, 37)) + [1029] + list(range(1030, len(items))):
        it = items[i]
        o, nb = descs[i]["out_off"], bins[i]
        r = oracle(1, it, traces[i], taps[i])
        assert np.linalg.norm(got[o:o + nb] - r) / np.linalg.norm(r) <= TOL, i
    o1, o2 = descs[-2]["out_off"], descs[-1]["out_off"]
    assert np.array_equal(got[o1:o1 + bins[-2]], got[o2:o2 + bins[-1]])
