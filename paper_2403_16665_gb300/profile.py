"""Run a named workload's forward transform a few times (for ncu / timing).

    python -m paper_2403_16665_gb300.profile --workload batch_r32 --batch 256 --iters 4

Inputs come from the seeded generators in signals.py; every iteration is one
full adfft_execute of the whole batch.  Prints the mean time per transform
from CUDA events.
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    import torch

    from paper_2403_16665_gb300 import _build, adfft, signals

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="batch_r32",
                    choices=["batch_r32", "batch_c64", "single_r64", "large_r32"])
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--alpha", type=float, default=None)
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--algo", type=int, default=adfft.ALGO_AUTO)
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--prec", type=int, default=adfft.PREC_NATIVE, help="0 native, 1 fp16x2, 2 bf16x3")
    args = ap.parse_args()
    _build.build()
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
    X = torch.empty((B, M), dtype=adfft.out_dtype(x.dtype), device=dev)
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
    nbytes = x.numel() * x.element_size() + B * M * X.element_size()
    print("workload=%s B=%d N=%d M=%d algo=%d fft_len=%d P=%d q=%d C=%d passes=%d prec=%d adjoint=%d  "
          "%.4f ms/transform  %.1f GB/s (input + output bytes)  %.3e points/s"
          % (args.workload, B, N, M, info.algo, info.fft_len, info.residues, info.fold, info.cluster, info.passes,
             args.prec, int(args.adjoint), ms, nbytes / ms / 1e6, B * M / ms * 1e3))


if __name__ == "__main__":
    main()
