"""Benchmark: batched spectral estimation of THz-TDS traces on one GB300.

A step is one pass of the whole hot path over one batch: the zero-padded FFT,
the chirp-z transform (Bluestein) and the Zoom FFT of every trace.  The
workload is 4096 synthetic traces of N = 2048 float32 samples at fs = 20 THz
(FFT to 16384, CZT 0.2-2.5 THz at M = 1024, Zoom FFT at 1.35 THz with D = 4
and a 63-tap Hamming low-pass), inputs resident in HBM.  The metric is
spectral bins per second (FFT N_FFT/2+1, CZT M, Zoom N_FFT/D bins per trace).

Timing: W warm-up steps, then K steps; before each step a 256 MB buffer is
written to flush L2 (outside the per-step events).  Every transform is
bracketed by CUDA events on the stream it runs on; the step time is the sum.
Multi-process (torchrun): each rank runs the same per-GPU batch (weak
scaling, no collective on the data path); the reported time is the max over
ranks and `value` counts the bins of all ranks.

``--impl reference`` times the FP64 CPU oracle instead (the reference arm of
this comparison): each step is a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2108_03948_gb300 import synth  # noqa: E402

METRIC = "spectral bins/s per transform at ≤1e-5 rel L2 vs FP64; % HBM/tensor roofline"
WORKLOAD = 1
# FP32 FMA peak: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest per-rank value (elapsed time) across the process group; the
    only cross-rank step of the benchmark (no collective on the data path)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bins_per_rank_step: int, steps: int, world: int, max_seconds: float) -> float:
    """Whole-job bins/s: every rank processes its own batch (weak scaling)."""
    return world * bins_per_rank_step * steps / max_seconds


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload_sizes(cfg):
    """Per-trace bins, algorithmic bytes and flops of each transform."""
    n = cfg.n
    L = max(16, 1 << (n + cfg.czt_m - 2).bit_length())
    K = cfg.zoom_n_fft // cfg.zoom_d
    lout = (n + cfg.zoom_taps - 1 + cfg.zoom_d - 1) // cfg.zoom_d
    return {
        "fft": {"bins": cfg.n_fft // 2 + 1, "bytes": 4 * n + 8 * (cfg.n_fft // 2 + 1),
                "flops": 2.5 * cfg.n_fft * np.log2(cfg.n_fft)},
        "czt": {"bins": cfg.czt_m, "bytes": 4 * n + 8 * cfg.czt_m,
                "flops": 2 * 5 * L * np.log2(L) + 6 * (n + L + cfg.czt_m)},
        "zoom": {"bins": K, "bytes": 4 * n + 8 * K,
                 "flops": 4 * lout * cfg.zoom_taps + 6 * n + 5 * K * np.log2(K)},
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path):
        self.path = path
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [s.strip() for s in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def oracle_sample(cfg, n_traces):
    """Time the FP64 oracle on the first n_traces of the workload.

    Returns (bins, seconds, outputs); this is the CPU-baseline leg, the only
    place the benchmark runs the oracle."""
    from oracle import spec_oracle as O
    x = synth.batch_traces(WORKLOAD, range(n_traces))
    taps = O.design_lowpass(cfg.zoom_taps, cfg.zoom_d)
    t0 = time.perf_counter()
    outs = {
        "fft": O.fft_padded(x, cfg.n_fft),
        "czt": O.czt(x, cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m),
        "zoom": O.zoom(x, cfg.fs, cfg.zoom_f1, cfg.zoom_f2, cfg.zoom_d, taps, cfg.zoom_n_fft),
    }
    dt = time.perf_counter() - t0
    bins = n_traces * (cfg.n_fft // 2 + 1 + cfg.czt_m + cfg.zoom_n_fft // cfg.zoom_d)
    return bins, dt, outs


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count() or 1


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    cfg = synth.UNIFORM[WORKLOAD]
    sample = 1024
    for _ in range(max(0, args.warmup)):
        oracle_sample(cfg, 16)
    times, bins_tot = [], 0
    for _ in range(args.steps):
        b, dt, _ = oracle_sample(cfg, sample)
        times.append(dt)
        bins_tot += b
    value = bins_tot / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "bins/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "4096 THz traces, N=2048, fs=20 THz; FFT 16384, CZT 0.2-2.5 THz M=1024, "
                               "Zoom 1.35 THz D=4 63 taps", "sample_traces_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "bins/s", "cores": cpu_threads(), "kind": "oracle",
                         "sample": f"{sample} of 4096 traces per step, all bins of all three transforms"},
        "e2e": {"value": value, "unit": "bins/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2108_03948_gb300 import spec

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = synth.UNIFORM[WORKLOAD]
    B = cfg.batch
    sizes = workload_sizes(cfg)
    x = synth.batch_traces(WORKLOAD, range(B))
    xd = torch.from_numpy(x).to(dev)
    taps_h = spec.spec_design_lowpass(cfg.zoom_taps, cfg.zoom_d)
    taps_d = torch.from_numpy(taps_h).to(dev)
    X = torch.empty((B, sizes["fft"]["bins"]), dtype=torch.complex64, device=dev)
    Z = torch.empty((B, sizes["czt"]["bins"]), dtype=torch.complex64, device=dev)
    U = torch.empty((B, sizes["zoom"]["bins"]), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ctx = spec.Context(local)
    stream = torch.cuda.current_stream(dev)

    def fft():
        spec.spec_fft(ctx, xd, cfg.fs, cfg.n_fft, out=X)

    def czt():
        spec.spec_czt(ctx, xd, cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m, out=Z)

    def zoom():
        spec.spec_zoom(ctx, xd, cfg.fs, cfg.zoom_f1, cfg.zoom_f2, cfg.zoom_d, taps_d, cfg.zoom_n_fft, out=U)

    parts = [("fft", fft), ("czt", czt), ("zoom", zoom)]
    for _ in range(max(3, args.warmup)):
        for _, f in parts:
            f()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    out_dir = os.path.join(ROOT, "gpurun_out")
    if not os.path.isdir(out_dir):
        import tempfile
        out_dir = tempfile.gettempdir()
    clocks = ClockSampler(local, os.path.join(out_dir, f"clocks_rank{rank}.csv"))
    with clocks:
        barrier()
        torch.cuda.synchronize()
        for s in range(args.steps):
            flush.zero_()
            evs[s][0].record(stream)
            for i, (_, f) in enumerate(parts):
                f()
                evs[s][i + 1].record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = args.steps * len(parts)
    per = {name: [evs[s][i].elapsed_time(evs[s][i + 1]) for s in range(args.steps)]
           for i, (name, _) in enumerate(parts)}
    step_ms = [sum(per[name][s] for name, _ in parts) for s in range(args.steps)]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    bins_step = B * sum(v["bins"] for v in sizes.values())
    value = job_throughput(bins_step, args.steps, world, total_ms / 1e3)

    # end to end through the C-ABI with host buffers (pinned), copies included
    xh = torch.from_numpy(x).pin_memory()
    Xh = torch.empty(X.shape, dtype=torch.complex64).pin_memory()
    Zh = torch.empty(Z.shape, dtype=torch.complex64).pin_memory()
    Uh = torch.empty(U.shape, dtype=torch.complex64).pin_memory()
    xn, Xn, Zn, Un = xh.numpy(), Xh.numpy(), Zh.numpy(), Uh.numpy()

    def e2e_step():
        spec.spec_fft(ctx, xn, cfg.fs, cfg.n_fft, out=Xn)
        spec.spec_czt(ctx, xn, cfg.fs, cfg.czt_f1, cfg.czt_f2, cfg.czt_m, out=Zn)
        spec.spec_zoom(ctx, xn, cfg.fs, cfg.zoom_f1, cfg.zoom_f2, cfg.zoom_d, taps_h, cfg.zoom_n_fft, out=Un)
    e2e_step()
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_val = job_throughput(bins_step, e2e_steps, world, e2e_s)
    h2d = 3 * x.nbytes + taps_h.nbytes
    d2h = X.numel() * 8 + Z.numel() * 8 + U.numel() * 8
    e2e_parity = max(float(np.abs(Xn - X.cpu().numpy()).max()), float(np.abs(Zn - Z.cpu().numpy()).max()),
                     float(np.abs(Un - U.cpu().numpy()).max()))

    if rank != 0:
        ctx.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    hbm, hbm_kind = measured_peaks()
    kern = {}
    for name in ("fft", "czt", "zoom"):
        ms = statistics.mean(per[name])
        gbs = B * sizes[name]["bytes"] / (ms / 1e3) / 1e9
        tfl = B * sizes[name]["flops"] / (ms / 1e3) / 1e12
        kern[name] = {"ms": ms, "bins_per_s": B * sizes[name]["bins"] / (ms / 1e3),
                      "hbm_gbs": gbs, "hbm_frac": gbs / hbm, "fp32_tflops": tfl,
                      "fp32_frac": tfl / FP32_PEAK_TFLOPS}
    dom = max(kern, key=lambda k: kern[k]["ms"])
    if kern[dom]["hbm_frac"] >= kern[dom]["fp32_frac"]:
        roof = {"bound": "hbm", "achieved": kern[dom]["hbm_gbs"], "peak": hbm, "unit": "GB/s",
                "frac": kern[dom]["hbm_frac"], "traffic": None, "kernel": dom,
                "peak_source": f"{hbm_kind} hbm_gbs"}
    else:
        roof = {"bound": "alu", "achieved": kern[dom]["fp32_tflops"], "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": kern[dom]["fp32_frac"], "traffic": None, "kernel": dom,
                "peak_source": "FP32 FMA 152 SM x 128 x 2 x 2.07 GHz"}
    traffic_file = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(traffic_file):
        with open(traffic_file) as f:
            tr = json.load(f).get(dom)
        if tr and tr.get("per_launch_bytes"):
            roof["traffic"] = tr["per_launch_bytes"]

    # CPU baseline leg (rank 0, N = 1 only): the FP64 oracle on the whole
    # batch, timed; its outputs also give the parity of the timed GPU outputs.
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        b, dt, ref = oracle_sample(cfg, B)
        cpu = {"value": b / dt, "unit": "bins/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"the whole batch ({B} traces), all bins of FFT, CZT and Zoom FFT, FP64 numpy, "
                         f"{dt:.1f} s"}
        for name, got in (("fft", X), ("czt", Z), ("zoom", U)):
            g = got.cpu().numpy().astype(np.complex128)
            r = ref[name]
            err = np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)
            kern[name]["max_rel_l2_all_traces"] = float(err.max())

    line = {
        "metric": METRIC, "value": value, "unit": "bins/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": statistics.mean(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "4096 THz traces, N=2048 float32, fs=20 THz; FFT to 16384, CZT 0.2-2.5 THz "
                               "M=1024, Zoom 1.35 THz D=4 63-tap Hamming; one launch per transform",
                   "batch_per_gpu": B, "l2": "flushed before every step (256 MB write)",
                   "bins_per_step_per_gpu": bins_step},
        "roofline": roof,
        "kernels": kern,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "bins/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps, "max_abs_diff_vs_device_path": e2e_parity},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
