"""Benchmark of the alpha-densified DFT on GB300.

One step = one forward transform (fold + twiddle + Stockham FFT + interleaved
epilogue, one kernel launch) of the whole batch: 4096 real fp32 signals,
N = 16384, alpha = 8, 131072 complex64 bins each (off-bin tones plus Gaussian
noise).  Inputs (256 MiB) and outputs (4 GiB) are far larger than the 129 MB
L2, so no flush is needed between timed steps.  Before warm-up the plan's launch
shape is chosen by the library's autotuner (adfft_plan_autotune, untimed).

    python bench.py [--gpus N --steps K --warmup W] [--impl native|reference]

For N > 1 (torchrun) every rank transforms its own batch (weak scaling, no
collective on the data path); the timed region is bracketed by barriers and
the max over ranks is reported.  --impl reference times the FP64 direct-sum
oracle on the host cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "α-dense spectrum points/s and % HBM roofline on 1 GB300 at stated error vs FP64"
UNIT = "points/s"
WORKLOAD = dict(workload="batch of 4096 real fp32 signals, N=16384, alpha=8 -> 131072 complex64 bins each",
                batch=4096, N=16384, alpha=8, M=131072, input="real fp32", output="complex64",
                signal="5 off-bin tones A~U(0.1,1) + white noise sigma=0.2, seed 2",
                l2="inputs 256 MiB + outputs 4 GiB > 129 MB L2; no flush between steps")
KERNEL_SOURCES = ["paper_2403_16665_gb300/csrc/fused.cuh", "paper_2403_16665_gb300/csrc/fft_device.cuh",
                  "paper_2403_16665_gb300/csrc/fused.cu"]


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kname, khash, shape):
    """dram read+write bytes per launch recorded from ncu for this exact kernel source and launch shape."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if (len(parts) >= 5 and not line.startswith("#") and parts[0] == kname and parts[1] == khash
                and parts[4] == shape):
            return float(parts[2])
    return None


def shape_tag(info):
    return "fft_len=%d,cluster=%d,staged=%d,grid=%d" % (info.fft_len, info.cluster, info.staged, info.grid)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        self.lines = []
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), power=float(f[3]), hw=f[5], hwt=f[6],
                                 swt=f[7], swpc=f[8]))
            except ValueError:
                continue
        if not rows:
            return None
        busy = [r for r in rows if r["power"] > 300.0] or rows
        reasons = set()
        for r in busy:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swpc", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r["sm"] for r in busy])),
                "sm_max_mhz": float(max(r["smax"] for r in rows)),
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(busy)}


def oracle_sample_rate(x, M, budget_s, rng):
    """Time the FP64 oracle on bounded bin samples of the workload: points/s."""
    import oracle
    nb = 64
    sig = 0
    t_total, pts = 0.0, 0
    while t_total < budget_s:
        bins = rng.integers(0, M, nb)
        t0 = time.perf_counter()
        oracle.alpha_dft(x[sig % x.shape[0]].astype(np.float64), M, bins=bins)
        dt = time.perf_counter() - t0
        t_total += dt
        pts += nb
        sig += 1
        if dt < budget_s / 20:
            nb *= 2
    return pts / t_total, pts, t_total


def run_reference(args):
    """Reference arm: the FP64 direct-sum oracle on the host cores (bounded samples)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2403_16665_gb300 import signals
    oracle.build()
    x, _ = signals.batch_r32(batch=4, N=WORKLOAD["N"], alpha=WORKLOAD["alpha"])
    M = WORKLOAD["M"]
    rng = np.random.default_rng(99)
    bins_per_step = 256
    for _ in range(args.warmup):
        oracle.alpha_dft(x[0].astype(np.float64), M, bins=rng.integers(0, M, 16))
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle.alpha_dft(x[s % 4].astype(np.float64), M, bins=rng.integers(0, M, bins_per_step))
    dt = time.perf_counter() - t0
    value = bins_per_step * args.steps / dt
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(WORKLOAD),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d bins per step of one signal (N=16384, M=131072), FP64 direct sum"
                                   % bins_per_step},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_native(args):
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_16665_gb300 import adfft, signals

    B, N, alpha, M = WORKLOAD["batch"], WORKLOAD["N"], WORKLOAD["alpha"], WORKLOAD["M"]
    x_np, _ = signals.batch_r32(batch=B, N=N, alpha=alpha, seed=2 + rank)
    x = torch.from_numpy(x_np).to(dev)
    X = torch.empty((B, M), dtype=torch.complex64, device=dev)
    plan = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    stream = torch.cuda.current_stream(dev)
    # launch shape chosen by the library's autotuner on this GPU (untimed set-up, like plan creation)
    if not args.no_tune:
        plan.autotune(x.data_ptr(), X.data_ptr(), stream, iters=5)
    info = plan.info

    def step():
        plan.execute(x.data_ptr(), X.data_ptr(), stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # error vs FP64 on sampled bins of a few signals (rank 0)
    err = None
    if rank == 0:
        import oracle
        rng = np.random.default_rng(5)
        sigs = np.array([0, B // 2, B - 1])
        bins = np.unique(rng.integers(0, M, 512))
        got = X[torch.from_numpy(sigs).to(dev)][:, torch.from_numpy(bins).to(dev)].cpu().numpy()
        ref = oracle.alpha_dft(x_np[sigs].astype(np.float64), M, bins=bins)
        e = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        err = {"rel_rms_max": float(e.max()), "tol": 2e-6 * np.log2(M),
               "sample": "3 signals x %d bins vs FP64 oracle" % bins.size}

    clocks = ClockSampler(dev.index)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    points = B * M * world
    value = points / (ms_per_step * 1e-3)

    # roofline of the fused kernel (the only kernel of a step)
    alg_bytes = B * N * 4 + B * M * 8
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (ms_per_step * 1e-3) / 1e9
    khash = kernel_hash()
    traffic = recorded_traffic("fused_forward_kernel", khash, shape_tag(info)) if info.passes == 1 else None

    # end to end through adfft_execute_host: pinned host input -> device -> spectrum -> host
    e2e = None
    if rank == 0 or world > 1:
        hx = torch.from_numpy(x_np).pin_memory()
        hX = torch.empty((B, M), dtype=torch.complex64).pin_memory()
        e2e_plan = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
        e2e_steps = max(1, min(args.steps, 5))
        e2e_plan.execute_host(hx.data_ptr(), hX.data_ptr(), stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_plan.execute_host(hx.data_ptr(), hX.data_ptr(), stream)
        dt = (time.perf_counter() - t0) / e2e_steps
        if world > 1:
            t = torch.tensor([dt], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": points / dt, "unit": UNIT, "h2d_bytes_per_step": B * N * 4,
               "d2h_bytes_per_step": B * M * 8, "ms_per_step": dt * 1e3, "steps": e2e_steps}
        e2e_plan.destroy()
        del hx, hX

    cpu = None
    if rank == 0:
        import oracle
        rate, pts, secs = oracle_sample_rate(x_np[:4], M, args.cpu_seconds, np.random.default_rng(7))
        cpu = {"value": rate, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
               "sample": "%d bins of 4 signals of the same workload, FP64 direct sum, %.1f s" % (pts, secs)}

    context = None
    if rank == 0 and not args.no_context:
        # the other configurations and cuFFT on zero-padded input, same GPU, outside the timed region
        from paper_2403_16665_gb300 import compare
        context = compare.context(dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(WORKLOAD, parallelism="independent replicas, one batch per GPU",
                           launch_shape={"algo": "fold" if info.passes == 1 else "four-step",
                                         "fft_len": info.fft_len, "residues": info.residues,
                                         "cluster": info.cluster, "staged": info.staged,
                                         "clusters_launched": info.grid, "autotuned": bool(info.tuned)}),
            "error_vs_fp64": err,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "fused_forward_kernel", "peak_kind": peak_kind,
                         "alg_bytes_per_launch": alg_bytes, "kernel_src_hash": khash},
            "cpu_baseline": cpu,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": args.steps * info.passes,
            "context": context,
        }
        print(json.dumps(line), flush=True)
    plan.destroy()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def free_port():
    import socket
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def spawn_ranks(n):
    """--gpus n > 1 without a torchrun environment: relaunch this command as n ranks (one
    per GPU, 127.0.0.1 rendezvous) and return the launcher's exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(n),
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-tune", action="store_true", help="keep the plan's default launch shape")
    ap.add_argument("--no-context", action="store_true",
                    help="skip the same-GPU measurements of the other configurations and of cuFFT")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.gpus < 1:
        ap.error("--gpus must be >= 1")
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        return spawn_ranks(args.gpus)
    world = dist_env()[0]
    if world != args.gpus and "WORLD_SIZE" in os.environ and "--gpus" in sys.argv:
        # the launcher's world size is what runs (and what n_gpus reports)
        print("bench.py: --gpus %d under WORLD_SIZE=%d; using %d ranks" % (args.gpus, world, world),
              file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
