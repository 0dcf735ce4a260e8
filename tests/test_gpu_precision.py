"""Precision forms: radix-16 stages on the tensor cores with split operands and
FP32 accumulation (FP16X2: fp16 hi + lo, 3 products; BF16X3: three bf16 parts, 6
products), against the FP64 oracle.  Every form is held to the FP32 tolerance
2e-6 * log2(M), overall and in every bin range of the large workload (windows
around the tones by amplitude decade, and the noise floor), for every signal
checked.  The errors are printed (pytest -s)."""
import numpy as np
import pytest

import oracle
from paper_2403_16665_gb300 import adfft, signals

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    adfft.load()
    return torch


BOUND = {adfft.PREC_NATIVE: 2e-6, adfft.PREC_FP16X2: 2e-6, adfft.PREC_BF16X3: 2e-6}


def run(torch, x_np, M, code, prec):
    dev = torch.device("cuda:0")
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(dev)
    B, N = x.shape
    plan = adfft.Plan(N, batch=B, dtype=code, M=M)
    plan.set_precision(prec)
    X = torch.empty((B, M), dtype=torch.complex64, device=dev)
    plan.execute(x.data_ptr(), X.data_ptr())
    plan.sync_status()
    return X, plan


@pytest.mark.parametrize("prec", [adfft.PREC_FP16X2, adfft.PREC_BF16X3])
@pytest.mark.parametrize("code,N,alpha", [(adfft.R32, 4096, 8), (adfft.C64, 8192, 2.5), (adfft.R32, 16384, 8),
                                          (adfft.C64, 2048, 3.75), (adfft.R32, 1 << 17, 8)])
def test_precision_forms_sampled(prec, code, N, alpha):
    torch = _torch()
    M = int(round(alpha * N))
    rng = np.random.default_rng(N)
    if code == adfft.R32:
        x = signals.batch_r32(batch=3, N=N, alpha=alpha)[0]
    else:
        x = signals.batch_c64(batch=3, N=N, alpha=alpha)[0]
    X, plan = run(torch, x, M, code, prec)
    bins = np.unique(np.concatenate([np.arange(16), rng.integers(0, M, 1500)]))
    got = X[:, torch.from_numpy(bins).cuda()].cpu().numpy()
    ref = oracle.alpha_dft(x.astype(np.complex128), M, bins=bins)
    err = (np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)).max()
    print("precision %d code %d N %d alpha %s passes %d: rel-RMS %.3e" % (prec, code, N, alpha, plan.info.passes, err))
    assert err <= BOUND[prec] * np.log2(M), err


def test_precision_rejected_where_unavailable():
    _torch()
    p64 = adfft.Plan(1024, batch=1, dtype=adfft.R64, M=4096)
    with pytest.raises(adfft.AdfftError):
        p64.set_precision(adfft.PREC_FP16X2)
    pz = adfft.Plan(1000, batch=1, dtype=adfft.C64, M=2500)     # chirp-z only
    with pytest.raises(adfft.AdfftError):
        pz.set_precision(adfft.PREC_BF16X3)


@pytest.mark.parametrize("prec", [adfft.PREC_NATIVE, adfft.PREC_FP16X2, adfft.PREC_BF16X3])
def test_large_precision_workload_per_bin_range(prec):
    """8 real fp32 signals, N = 2^22, alpha = 16: error per bin range (windows of
    +-2 alpha bins around tones grouped by amplitude decade, and the rest)."""
    torch = _torch()
    x, prm = signals.large_r32(batch=2)
    N, M = 1 << 22, 1 << 26
    X, plan = run(torch, x, M, adfft.R32, prec)
    rng = np.random.default_rng(4)
    tol = BOUND[prec] * np.log2(M)
    for s in range(x.shape[0]):
        A, nu = prm["A"][s], prm["nu"][s]
        groups = {}
        for a_lo in (1e-4, 1e-3, 1e-2, 1e-1):
            sel = (A >= a_lo) & (A < 10 * a_lo)
            if not sel.any():
                continue
            centers = np.round(nu[sel] * 16).astype(np.int64)
            win = (centers[:, None] + np.arange(-32, 33)[None, :]).ravel() % M
            groups["tones %.0e..%.0e" % (a_lo, 10 * a_lo)] = np.unique(win)
        groups["noise floor"] = np.unique(rng.integers(0, M, 400))
        allbins = np.unique(np.concatenate(list(groups.values())))
        got_all = X[s, torch.from_numpy(allbins).cuda()].cpu().numpy()
        ref_all = oracle.alpha_dft(x[s].astype(np.float64), M, bins=allbins)
        pos = {b: i for i, b in enumerate(allbins)}
        report, errs = [], {}
        for name, b in groups.items():
            idx = np.array([pos[v] for v in b])
            e = np.linalg.norm(got_all[idx] - ref_all[idx]) / np.linalg.norm(ref_all[idx])
            errs[name] = e
            report.append("%s: %.2e" % (name, e))
        overall = np.linalg.norm(got_all - ref_all) / np.linalg.norm(ref_all)
        print("precision %d, N=2^22 alpha=16, signal %d, rel-RMS overall %.2e; %s"
              % (prec, s, overall, "; ".join(report)))
        assert np.isfinite(got_all).all()
        assert overall <= tol, (s, overall)
        for name, e in errs.items():
            assert e <= tol, (s, name, e)
