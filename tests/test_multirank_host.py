"""Multi-GPU host logic on CPU: the trace partition (every trace exactly once,
cost-balanced ragged shares, order restored on gather) and the benchmark's
cross-rank timing, with two gloo ranks.  Traces are independent sums (Section
2.1, Eq. 2; Section 2.3, Eq. 11), so a partition by trace is exact."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2108_03948_gb300 import shard, synth  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(target, world, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q, *args)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def _timing_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.0 + rank, world)          # rank 1 is slower
    bins = bench.sum_over_ranks(1000 * (rank + 1), world)
    v = bench.job_throughput(bins, 10, t)
    q.put((rank, t, bins, v))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    res = _spawn(_timing_worker, 2)
    assert [r[1] for r in res] == [2.0, 2.0]
    assert [r[2] for r in res] == [3000.0, 3000.0]
    assert all(abs(r[3] - 3000 * 10 / 2.0) < 1e-9 for r in res)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.sum_over_ranks(7, 1) == 7.0
    assert bench.job_throughput(100, 4, 2.0) == 200.0


@pytest.mark.parametrize("total,world", [(0, 3), (1, 2), (4096, 2), (4097, 8), (65536, 8), (256, 3)])
def test_contiguous_slices_cover_every_trace_once(total, world):
    sl = shard.contiguous_slices(total, world)
    assert len(sl) == world
    flat = [i for a, b in sl for i in range(a, b)]
    assert flat == list(range(total))
    sizes = [b - a for a, b in sl]
    assert max(sizes) - min(sizes) <= 1


def _ragged_costs(count):
    rg = synth.ragged_params(count)
    return [shard.ragged_trace_cost(it.n, it.n_fft, it.m, it.d, it.n_taps) for it in rg.items]


@pytest.mark.parametrize("world", [2, 4, 8])
def test_ragged_split_is_a_partition_within_ten_percent(world):
    costs = _ragged_costs(10000)
    parts = shard.balance_by_cost(costs, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(10000))
    assert all(p == sorted(p) for p in parts)
    assert shard.imbalance(costs, parts) <= 0.10
    # much better than a naive contiguous split of the same list
    naive = shard.slices_as_parts(shard.contiguous_slices(10000, world))
    assert shard.imbalance(costs, parts) <= shard.imbalance(costs, naive)


def test_cost_model_orders_the_work():
    # a longer trace, a larger Bluestein length or more zoom bins never costs less
    base = shard.ragged_trace_cost(2000, 16384, 1024, 4, 63)
    assert shard.ragged_trace_cost(4000, 32768, 1024, 4, 63) > base
    assert shard.ragged_trace_cost(2000, 16384, 4096, 4, 63) > base
    assert shard.ragged_trace_cost(2000, 16384, 1024, 2, 63) > base


def test_assemble_rejects_overlap_and_gaps():
    with pytest.raises(ValueError):
        shard.assemble([[0, 1], [1]], [["a", "b"], ["c"]], 2)
    with pytest.raises(ValueError):
        shard.assemble([[0], [2]], [["a"], ["c"]], 3)
    assert shard.assemble([[1], [0, 2]], [["b"], ["a", "c"]], 3) == ["a", "b", "c"]


def _spectrum_stand_in(trace, n_fft):
    """A per-trace result computed on the CPU: 16 bins of the oracle's padded
    FFT (the partition logic only needs a result that depends on the trace)."""
    from oracle import spec_oracle as O
    bins = np.linspace(0, n_fft // 2, 16).round().astype(np.int64)
    return O.fft_padded_bins(trace, n_fft, bins)[0]


def _gather_worker(rank, world, port, q, count):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rg = synth.ragged_params(count)
    costs = [shard.ragged_trace_cost(it.n, it.n_fft, it.m, it.d, it.n_taps) for it in rg.items]
    parts = shard.balance_by_cost(costs, world)
    mine = [_spectrum_stand_in(synth.ragged_trace(i, rg.items[i]), rg.items[i].n_fft) for i in parts[rank]]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    whole = shard.assemble(parts, gathered, count)
    # uniform workload: contiguous slices of workload 1's traces
    sl = shard.contiguous_slices(10, world)
    a, b = sl[rank]
    x = synth.batch_traces(1, range(a, b), n=64)
    u_mine = [_spectrum_stand_in(x[j], 256) for j in range(b - a)]
    u_gathered = [None] * world
    dist.all_gather_object(u_gathered, u_mine)
    u_whole = shard.assemble(shard.slices_as_parts(sl), u_gathered, 10)
    q.put((rank, whole, u_whole))
    dist.destroy_process_group()


def test_gathered_spectra_match_the_single_rank_order():
    count = 24
    res = _spawn(_gather_worker, 2, count)
    rg = synth.ragged_params(count)
    single = [_spectrum_stand_in(synth.ragged_trace(i, rg.items[i]), rg.items[i].n_fft) for i in range(count)]
    x = synth.batch_traces(1, range(10), n=64)
    u_single = [_spectrum_stand_in(x[j], 256) for j in range(10)]
    for _, whole, u_whole in res:
        assert len(whole) == count
        for a, b in zip(whole, single):
            np.testing.assert_array_equal(a, b)
        for a, b in zip(u_whole, u_single):
            np.testing.assert_array_equal(a, b)


def test_bench_rank_share_weak_and_strong():
    import bench
    w0, tot = bench.rank_share(1, 0, 2, "weak")
    w1, _ = bench.rank_share(1, 1, 2, "weak")
    assert tot == 8192 and w0 == list(range(4096)) and w1 == list(range(4096, 8192))
    s0, tot_s = bench.rank_share(1, 0, 2, "strong")
    s1, _ = bench.rank_share(1, 1, 2, "strong")
    assert tot_s == 4096 and s0 + s1 == list(range(4096))


def test_bench_gpus_n_starts_n_ranks_itself(monkeypatch):
    import bench
    seen = {}

    def fake_call(cmd):
        seen["cmd"] = cmd
        return 0
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(bench.subprocess, "call", fake_call)
    assert bench.main(["--gpus", "4", "--steps", "3", "--warmup", "3"]) == 0
    cmd = seen["cmd"]
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and "--master-addr=127.0.0.1" in cmd
    assert cmd[-6:] == ["--gpus", "4", "--steps", "3", "--warmup", "3"]
