"""Same-GPU context measurements for the benchmark line (not part of the transform).

For every workload of the five configurations this times the library's forward
transform (and, where it has one, the adjoint and the precision forms) on the
seeded synthetic inputs of signals.py, and, as the comparison the paper's
method is measured against (the zero-padding equivalence of Sec. 2 and the
cost argument of Sec. 4, Eq. 16), cuFFT on the input zero-padded to M points
through torch.fft, with the padding included in its time.  cuFFT runs here
only; the library never calls it.  Accuracy against the FP64 oracle is given
on sampled bins for every form timed (cuFFT's output scaled by S = 1/N, the
library's default scale).  The ragged batch is timed as the class graph (forward, adjoint)
and as one persistent work-queue kernel (forward), with the two forwards' difference.
"""
from __future__ import annotations

import time

import numpy as np


def _time(fn, iters, warm=2):
    import torch
    s = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(iters):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / max(1, iters)


def _err(got, ref):
    return float((np.linalg.norm(got - ref, axis=-1) / np.linalg.norm(ref, axis=-1)).max())


def _entry(ms, points, nbytes, err=None, **kw):
    d = {"ms": round(ms, 5), "points_per_s": points / ms * 1e3, "gbs": nbytes / ms / 1e6}
    if err is not None:
        d["rel_rms_vs_fp64"] = err
    d.update(kw)
    return d


def _sample_err(torch, X, x_np, M, sigs, nbins, seed, scale=1.0, centers=None):
    """rel-RMS against the oracle over random bins plus, where the spectrum is peaky (tones far
    above the noise), windows of +-32 bins around the tone bins `centers`: random bins alone
    would miss the bins that hold most of the energy and overstate the relative error."""
    import oracle
    rng = np.random.default_rng(seed)
    bins = rng.integers(0, M, nbins)
    if centers is not None:
        bins = np.concatenate([bins, (np.asarray(centers)[:, None] + np.arange(-32, 33)[None, :]).ravel() % M])
    bins = np.unique(bins)
    got = X[torch.tensor(sigs, device=X.device)][:, torch.from_numpy(bins).to(X.device)].cpu().numpy() * scale
    x = x_np[sigs]
    ref = oracle.alpha_dft(x.astype(np.complex128 if np.iscomplexobj(x) else np.float64), M, bins=bins)
    return _err(got, ref)


def cufft_padded(torch, x, M, real, iters=5, with_c2c=True):
    """cuFFT of the input zero-padded to M points: C2C of the padded complex signal (all M
    bins) and, for real input, R2C (M/2 + 1 bins).  Padding inside the timed region."""
    B, N = x.shape
    out = {}

    def c2c():
        xc = torch.zeros((B, M), dtype=torch.complex64, device=x.device)
        xc[:, :N] = x
        return torch.fft.fft(xc, dim=1)
    in_b = B * N * x.element_size()
    if with_c2c:
        ms = _time(c2c, iters)
        out["c2c_padded"] = _entry(ms, B * M, in_b + B * M * 8, note="all M bins, pad included, unscaled")
    if real:
        ms = _time(lambda: torch.fft.rfft(x, n=M, dim=1), iters)
        out["r2c_padded"] = _entry(ms, B * (M // 2 + 1), in_b + B * (M // 2 + 1) * 8,
                                   note="M/2+1 bins (half spectrum), pad included, unscaled")
    return out, c2c


def context(dev, iters=5, seed_bins=11):
    """Measurements of every configuration on the current GPU (a dict for the JSON line)."""
    import torch

    from paper_2403_16665_gb300 import adfft, signals

    res = {}
    t_start = time.time()

    # single real fp64 signal, N = 1024, alpha = 4 (launch-bound)
    try:
        x_np, _ = signals.single_r64()
        x = torch.from_numpy(x_np).to(dev)
        M = 4096
        plan = adfft.Plan(1024, batch=1, dtype=adfft.R64, M=M)
        X = torch.empty((1, M), dtype=torch.complex128, device=dev)
        ms = _time(lambda: plan.execute(x.data_ptr(), X.data_ptr()), 50)
        res["single_r64_N1024_a4"] = _entry(ms, M, 1024 * 8 + M * 16,
                                            _sample_err(torch, X, x_np, M, [0], 512, seed_bins))
    except Exception as e:   # context only: report, never fail the benchmark
        res["single_r64_N1024_a4"] = {"error": repr(e)[:200]}

    # 4096 real fp32, N = 16384, alpha = 8: cuFFT on the zero-padded input
    try:
        x_np, _ = signals.batch_r32(batch=4096, N=16384, alpha=8)
        x = torch.from_numpy(x_np).to(dev)
        M = 131072
        cu, c2c = cufft_padded(torch, x, M, True, iters)
        Xc = c2c()
        cu["c2c_padded"]["rel_rms_vs_fp64"] = _sample_err(torch, Xc, x_np, M, [0, 4095], 512, seed_bins,
                                                          scale=1.0 / 16384)
        del Xc
        res["batch_r32_4096_N16384_a8"] = {"cufft": cu}
        del x
        torch.cuda.empty_cache()
    except Exception as e:
        res["batch_r32_4096_N16384_a8"] = {"error": repr(e)[:200]}

    # 1024 complex64, N = 8192, alpha 2.5 / 3.75: fold form, chirp-z form, cuFFT
    for alpha in (2.5, 3.75):
        key = "batch_c64_1024_N8192_a%s" % alpha
        try:
            x_np, _ = signals.batch_c64(batch=1024, N=8192, alpha=alpha)
            x = torch.from_numpy(x_np).to(dev)
            M = int(round(alpha * 8192))
            nbytes = x.numel() * 8 + 1024 * M * 8
            d = {}
            for name, algo in (("fold", adfft.ALGO_FOLD), ("chirp_z", adfft.ALGO_BLUESTEIN)):
                plan = adfft.Plan(8192, batch=1024, dtype=adfft.C64, M=M)
                X = torch.empty((1024, M), dtype=torch.complex64, device=dev)
                if algo == adfft.ALGO_FOLD:
                    # launch shape from the autotuner (untimed set-up, as the benchmark does)
                    plan.autotune(x.data_ptr(), X.data_ptr(), iters=3)
                    d["fold_launch_shape"] = {"fft_len": plan.info.fft_len, "cluster": plan.info.cluster,
                                              "staged": plan.info.staged, "algo": plan.info.algo}
                plan.set_algorithm(algo)
                ms = _time(lambda: plan.execute(x.data_ptr(), X.data_ptr()), iters)
                d[name] = _entry(ms, 1024 * M, nbytes, _sample_err(torch, X, x_np, M, [0, 1023], 256, seed_bins))
            cu, c2c = cufft_padded(torch, x, M, False, iters)
            Xc = c2c()
            cu["c2c_padded"]["rel_rms_vs_fp64"] = _sample_err(torch, Xc, x_np, M, [0, 1023], 256, seed_bins,
                                                              scale=1.0 / 8192)
            d["cufft"] = cu
            res[key] = d
            del X, Xc, x
        except Exception as e:
            res[key] = {"error": repr(e)[:200]}
    torch.cuda.empty_cache()

    # 8 real fp32, N = 2^22, alpha = 16: FP32 form, precision forms, adjoint, cuFFT
    try:
        x_np, prm = signals.large_r32(batch=8)
        centers = np.round(prm["nu"][0] * 16).astype(np.int64)
        x = torch.from_numpy(x_np).to(dev)
        N, M = 1 << 22, 1 << 26
        nbytes = x.numel() * 4 + 8 * M * 8
        X = torch.empty((8, M), dtype=torch.complex64, device=dev)
        d = {}
        for name, prec in (("fp32", adfft.PREC_NATIVE), ("fp16x2", adfft.PREC_FP16X2),
                           ("bf16x3", adfft.PREC_BF16X3)):
            plan = adfft.Plan(N, batch=8, dtype=adfft.R32, M=M)
            if prec == adfft.PREC_NATIVE:
                # split Nc = A B from the autotuner (untimed set-up)
                plan.autotune(x.data_ptr(), X.data_ptr(), iters=2)
                d["fp32_launch_shape"] = {"algo": plan.info.algo, "four_step_a": plan.info.four_step_a,
                                          "cluster": plan.info.cluster}
            plan.set_precision(prec)
            ms = _time(lambda: plan.execute(x.data_ptr(), X.data_ptr()), 3, warm=1)
            d[name] = _entry(ms, 8 * M, nbytes, _sample_err(torch, X, x_np, M, [0], 96, seed_bins, centers=centers))
            if prec == adfft.PREC_NATIVE:
                xb = torch.empty_like(x)
                ms = _time(lambda: plan.execute_adjoint(X.data_ptr(), xb.data_ptr()), 3, warm=1)
                d["fp32_adjoint"] = _entry(ms, 8 * M, nbytes)
                del xb
        del X
        torch.cuda.empty_cache()
        cu, _ = cufft_padded(torch, x, M, True, 3, with_c2c=False)   # R2C only at this size
        d["cufft"] = cu
        res["large_r32_8_N2p22_a16"] = d
        del x
        torch.cuda.empty_cache()
    except Exception as e:
        res["large_r32_8_N2p22_a16"] = {"error": repr(e)[:200]}

    # 10000 ragged real fp32 signals: forward and adjoint (graph replays)
    try:
        x_np, Ns, alphas, _ = signals.ragged_r32(count=10000)
        plan = adfft.RaggedPlan(Ns, alphas, adfft.R32)
        x = torch.from_numpy(x_np).to(dev)
        X = torch.empty(int(plan.out_off[-1]), dtype=torch.complex64, device=dev)
        xb = torch.empty_like(x)
        nbytes = x.numel() * 4 + X.numel() * 8
        ms = _time(lambda: plan.execute(x.data_ptr(), X.data_ptr()), iters)
        d = {"forward": _entry(ms, X.numel(), nbytes)}
        ms = _time(lambda: plan.execute_adjoint(X.data_ptr(), xb.data_ptr()), iters)
        d["adjoint"] = _entry(ms, X.numel(), nbytes)
        try:
            # the same forward as one persistent work-queue kernel, against the class graph
            Xq = torch.empty_like(X)
            plan.set_form(adfft.RAGGED_QUEUE)
            ms = _time(lambda: plan.execute(x.data_ptr(), Xq.data_ptr()), iters)
            plan.set_form(adfft.RAGGED_CLASSES)
            plan.execute(x.data_ptr(), X.data_ptr())
            torch.cuda.synchronize()
            rel = (torch.linalg.vector_norm(Xq - X) / torch.linalg.vector_norm(X)).item()
            d["queue_forward"] = _entry(ms, X.numel(), nbytes, rel_diff_vs_class_graph=rel)
            del Xq
        except Exception as e:
            d["queue_forward"] = {"error": repr(e)[:200]}
        res["ragged_r32_10000"] = d
        del x, X, xb
        torch.cuda.empty_cache()
    except Exception as e:
        res["ragged_r32_10000"] = {"error": repr(e)[:200]}
    res["seconds"] = round(time.time() - t_start, 1)
    return res
