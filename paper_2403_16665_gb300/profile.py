"""Run a named workload's forward transform a few times (for ncu / timing).

    python -m paper_2403_16665_gb300.profile --workload batch_r32 --batch 256 --iters 4
    python -m paper_2403_16665_gb300.profile --workload ragged_r32 --batch 10000 --iters 10
    python -m paper_2403_16665_gb300.profile --workload ragged_r32 --batch 10000 --iters 10 --subsets
    python -m paper_2403_16665_gb300.profile --probes [write|dsmem|overlap|l2|place]

Inputs come from the seeded generators in signals.py; every iteration is one
full adfft_execute of the whole batch.  Prints the mean time per transform
from CUDA events.  The ragged workload is timed three ways: the ragged plan
(one graph replay per execute, forward and adjoint), one uniform plan per
shape class executed one after another, and one execute per signal.
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    import torch

    from paper_2403_16665_gb300 import _build, adfft, signals

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="batch_r32",
                    choices=["batch_r32", "batch_c64", "single_r64", "large_r32", "ragged_r32"])
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--alpha", type=float, default=None)
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--algo", type=int, default=adfft.ALGO_AUTO)
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--prec", type=int, default=adfft.PREC_NATIVE, help="0 native, 1 fp16x2, 2 bf16x3")
    ap.add_argument("--tune", action="store_true", help="autotune the plan first (adfft_plan_autotune)")
    ap.add_argument("--shape", default=None,
                    help="fold launch shape fft_len,cluster,staged[,grid] (adfft_plan_set_launch_shape)")
    ap.add_argument("--half", action="store_true", help="half-spectrum output (real input: bins 0 .. M/2)")
    ap.add_argument("--subsets", action="store_true",
                    help="ragged_r32: class graph against the queue form on subsets of the mix")
    ap.add_argument("--probes", nargs="?", const="all", default=None,
                    help="build and run the exchange-path micro-benchmarks (write, dsmem, overlap, l2, "
                         "place or all) instead of a workload")
    args = ap.parse_args()
    if args.probes:
        return probes(args.probes)
    _build.build()
    if args.workload == "ragged_r32":
        return ragged_subsets(args) if args.subsets else ragged(args)
    gen = getattr(signals, args.workload)
    kw = dict(batch=args.batch)
    if args.N:
        kw["N"] = args.N
    if args.alpha:
        kw["alpha"] = args.alpha
    x_np, _ = gen(**kw)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(x_np).to(dev)
    B, N = x.shape
    alpha = args.alpha or {"batch_r32": 8, "batch_c64": 2.5, "single_r64": 4, "large_r32": 16}[args.workload]
    M = int(round(alpha * N))
    dt = {np.dtype(np.float32): adfft.R32, np.dtype(np.complex64): adfft.C64,
          np.dtype(np.float64): adfft.R64, np.dtype(np.complex128): adfft.C128}[x_np.dtype]
    plan = adfft.Plan(N, batch=B, dtype=dt, M=M)
    if args.algo != adfft.ALGO_AUTO:
        plan.set_algorithm(args.algo)
    if args.prec != adfft.PREC_NATIVE:
        plan.set_precision(args.prec)
    if args.half:
        plan.set_output(adfft.OUTPUT_HALF)
    X = torch.empty((B, plan.info.out_bins), dtype=adfft.out_dtype(x.dtype), device=dev)
    if args.shape:
        plan.set_launch_shape(*(int(v) for v in args.shape.split(",")))
    if args.tune:
        # with --adjoint the tuner times forward + adjoint steps (the adjoint's output overwrites x)
        plan.autotune(x.data_ptr(), X.data_ptr(), with_adjoint=args.adjoint)
    g = torch.empty_like(x) if args.adjoint else None
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(args.iters + 1):
        if i == 1:
            e0.record(s)
        if args.adjoint:
            plan.execute_adjoint(X.data_ptr(), g.data_ptr(), s)
        else:
            plan.execute(x.data_ptr(), X.data_ptr(), s)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.iters)
    info = plan.info
    nbytes = x.numel() * x.element_size() + X.numel() * X.element_size()
    print("workload=%s B=%d N=%d M=%d algo=%d fft_len=%d A=%d P=%d q=%d C=%d staged=%d grid=%d tuned=%d passes=%d "
          "prec=%d adjoint=%d  "
          "%.4f ms/transform  %.1f GB/s (input + output bytes)  %.3e points/s"
          % (args.workload, B, N, M, info.algo, info.fft_len, info.four_step_a, info.residues, info.fold,
             info.cluster, info.staged, info.grid, info.tuned, info.passes,
             args.prec, int(args.adjoint), ms, nbytes / ms / 1e6, B * M / ms * 1e3))


def probes(which):
    """Compile probes/exchange_probes.cu for sm_103a next to the library and run it."""
    import os
    import subprocess

    from paper_2403_16665_gb300 import _build
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "probes", "exchange_probes.cu")
    exe = os.path.join(_build.LIBDIR, "exchange_probes")
    os.makedirs(_build.LIBDIR, exist_ok=True)
    subprocess.run([_build.nvcc(), *_build.ARCH, "-O3", "-std=c++17", "-o", exe, src], check=True)
    return subprocess.run([exe, which]).returncode


def _time(fn, iters):
    import torch
    s = torch.cuda.current_stream()
    fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(iters):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / max(1, iters)


def ragged_subsets(args):
    """Forward of the class graph and of the queue form on subsets of the ragged mix (a ragged
    plan built from each subset's signals, random input)."""
    import torch

    from paper_2403_16665_gb300 import adfft, signals

    Ns, alphas = signals.ragged_shapes(args.batch)
    Ms = np.rint(Ns * alphas).astype(np.int64)
    dev = torch.device("cuda:0")
    subsets = [("all", np.ones(len(Ns), bool)), ("M > 32768", Ms > 32768), ("M <= 32768", Ms <= 32768),
               ("N = 65536, M = 524288", (Ns == 65536) & (Ms == 524288)), ("N = 16384", Ns == 16384),
               ("N <= 2048", Ns <= 2048)]
    for name, sel in subsets:
        plan = adfft.RaggedPlan(Ns[sel], alphas[sel], adfft.R32)
        x = torch.randn(int(plan.in_off[-1]), device=dev)
        X = torch.empty(int(plan.out_off[-1]), dtype=torch.complex64, device=dev)
        nbytes = x.numel() * 4 + X.numel() * 8
        plan.set_form(adfft.RAGGED_CLASSES)
        tg = _time(lambda: plan.execute(x.data_ptr(), X.data_ptr()), args.iters)
        try:
            plan.set_form(adfft.RAGGED_QUEUE)
            tq = _time(lambda: plan.execute(x.data_ptr(), X.data_ptr()), args.iters)
        except adfft.AdfftError:
            tq = float("nan")
        print("ragged subset %-24s signals %5d  %.3f GB  class graph %.4f ms (%.0f GB/s)  queue %.4f ms (%.0f GB/s)"
              % (name, int(sel.sum()), nbytes / 1e9, tg, nbytes / tg / 1e6, tq, nbytes / tq / 1e6))


def ragged(args):
    import torch

    from paper_2403_16665_gb300 import adfft, signals

    x_np, Ns, alphas, _ = signals.ragged_r32(count=args.batch)
    dev = torch.device("cuda:0")
    plan = adfft.RaggedPlan(Ns, alphas, adfft.R32)
    in_off, out_off = plan.in_off, plan.out_off
    x = torch.from_numpy(x_np).to(dev)
    X = torch.empty(int(out_off[-1]), dtype=torch.complex64, device=dev)
    g = torch.randn(int(out_off[-1]), dtype=torch.complex64, device=dev)
    xb = torch.empty_like(x)
    nbytes = x.numel() * 4 + X.numel() * 8
    points = X.numel()
    peak = None
    try:
        import json
        import os
        with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                               "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["hbm_gbs"])
    except Exception:
        pass

    def report(name, ms):
        gbs = nbytes / ms / 1e6
        frac = (" %.1f%% of measured HBM" % (100 * gbs / peak)) if peak else ""
        print("ragged count=%d %-34s %.4f ms  %.1f GB/s%s  %.3e points/s"
              % (len(Ns), name, ms, gbs, frac, points / ms * 1e3))

    report("ragged plan, forward", _time(lambda: plan.execute(x.data_ptr(), X.data_ptr()), args.iters))
    try:
        plan.set_form(adfft.RAGGED_QUEUE)
        Xq = torch.empty_like(X)
        report("ragged plan, forward, queue form", _time(lambda: plan.execute(x.data_ptr(), Xq.data_ptr()), args.iters))
        plan.set_form(adfft.RAGGED_CLASSES)
        plan.execute(x.data_ptr(), X.data_ptr())
        torch.cuda.synchronize()
        print("queue form vs class graph: rel difference %.2e"
              % (torch.linalg.norm(Xq - X) / torch.linalg.norm(X)).item())
        del Xq
    except adfft.AdfftError as e:
        print("queue form not available:", e)
    report("ragged plan, adjoint", _time(lambda: plan.execute_adjoint(g.data_ptr(), xb.data_ptr()), args.iters))
    Xr = X.clone()
    if args.tune:
        Xt = torch.empty_like(X)
        plan.autotune(x.data_ptr(), Xt.data_ptr(), with_adjoint=True)
        report("ragged plan, tuned (fwd + adj), forward", _time(lambda: plan.execute(x.data_ptr(), Xt.data_ptr()), args.iters))
        report("ragged plan, tuned (fwd + adj), adjoint",
               _time(lambda: plan.execute_adjoint(g.data_ptr(), xb.data_ptr()), args.iters))
        d = (torch.linalg.norm(Xt - Xr) / torch.linalg.norm(Xr)).item()
        print("ragged tuned vs untuned forward: rel difference %.2e" % d)
    # one uniform plan per shape class, run one after another on one stream
    Ms = np.rint(alphas * Ns).astype(np.int64)
    classes = {}
    for i, (n, m) in enumerate(zip(Ns.tolist(), Ms.tolist())):
        classes.setdefault((n, m), []).append(i)
    runs = []
    for (n, m), idx in sorted(classes.items()):
        idx_t = torch.tensor(idx)
        xi = torch.stack([x[int(in_off[i]):int(in_off[i + 1])] for i in idx])
        Xi = torch.empty((len(idx), m), dtype=torch.complex64, device=dev)
        p = adfft.Plan(n, batch=len(idx), dtype=adfft.R32, M=m)
        runs.append((p, xi, Xi, idx_t))
    report("uniform plan per class (%d)" % len(runs),
           _time(lambda: [p.execute(xi.data_ptr(), Xi.data_ptr()) for p, xi, Xi, _ in runs], args.iters))
    # per-class times (each class alone, uniform plan), slowest first
    rows = []
    for p, xi, Xi, idx in runs:
        ms = _time(lambda: p.execute(xi.data_ptr(), Xi.data_ptr()), args.iters)
        i = p.info
        b = xi.numel() * 4 + Xi.numel() * 8
        rows.append((ms, int(i.N), int(i.M), len(idx), b, i))
        for k, j in enumerate(idx.tolist()):
            ref = Xr[int(out_off[j]):int(out_off[j + 1])]
            d = (torch.linalg.norm(Xi[k] - ref) / torch.linalg.norm(ref)).item()
            if d > 1e-6:
                raise SystemExit("per-class result differs from the ragged plan at signal %d: %.2e" % (j, d))
    rows.sort(key=lambda r: -r[0])
    total = sum(r[0] for r in rows)
    print("per class (alone): N M count  ms  share  GB/s  algo fft_len P q C staged tuned")
    for ms, n, m, cnt, b, i in rows:
        print("  %6d %7d %5d  %.4f  %4.1f%%  %7.1f  %d %d %d %d %d %d %d"
              % (n, m, cnt, ms, 100 * ms / total, b / ms / 1e6, i.algo, i.fft_len, i.residues, i.fold,
                 i.cluster, i.staged, i.tuned))
    # one execute per signal, batch-1 plans on the packed buffers
    single = {key: adfft.Plan(key[0], batch=1, dtype=adfft.R32, M=key[1]) for key in classes}
    xp, Xp = x.data_ptr(), X.data_ptr()
    calls = [(single[(n, m)], xp + 4 * int(in_off[i]), Xp + 8 * int(out_off[i]))
             for i, (n, m) in enumerate(zip(Ns.tolist(), Ms.tolist()))]
    report("one execute per signal", _time(lambda: [p.execute(a, b) for p, a, b in calls], max(1, args.iters // 5)))
    d = (torch.linalg.norm(X - Xr) / torch.linalg.norm(Xr)).item()
    if d > 1e-6:
        raise SystemExit("per-signal result differs from the ragged plan: %.2e" % d)


if __name__ == "__main__":
    import sys
    sys.exit(main())
