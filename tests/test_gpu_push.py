"""GPU parity of the push-exchange forward kernel (clusters of 8 CTAs, one residue each,
runs exchanged by bulk copies) on the 16384-sample, alpha = 8 real fp32 class.

Against the FP64 oracle on contiguous bin blocks that straddle every CTA's output
ranges (direct bins j and j + Mc, mirror bins Mc - j and M - j), the half boundaries
of each range, and random bins, for several signals of the persistent grid; against
the peer-load (pull) epilogue of the same plan at every bin.
Tolerance: relative RMS per signal <= 2e-6 * log2(M) (FP32 forms).
"""
import numpy as np
import pytest

import oracle
from paper_2403_16665_gb300 import adfft, signals

pytestmark = pytest.mark.gpu

N, ALPHA = 16384, 8
M = N * ALPHA
Mc = M // 2
JC = N // 4            # leader bins per CTA: Np / 2 with the packed sub-FFT Np = N / 2
TOL = 2e-6 * np.log2(M)


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    adfft.load()
    return torch


def boundary_bins():
    """Blocks of 48 bins around every range start of every CTA and half, all four ranges."""
    edges = set()
    for c in range(9):
        for h in (0, 0.5):
            j = int(JC * (c + h))
            for e in (j, Mc + j, Mc - j, M - j):
                edges.add(e)
    bins = set()
    for e in edges:
        for b in range(e - 24, e + 24):
            if 0 <= b < M:
                bins.add(b)
    rng = np.random.default_rng(3)
    bins.update(rng.integers(0, M, 512).tolist())
    return np.array(sorted(bins), dtype=np.int64)


def run(torch, x, staged, batch_grid=0):
    B = x.shape[0]
    plan = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    plan.set_launch_shape(N // 2, 8, staged, batch_grid)
    info = plan.info
    X = torch.empty((B, M), dtype=torch.complex64, device=x.device)
    plan.execute(x.data_ptr(), X.data_ptr())
    plan.sync_status()   # raises if a bounded wait of the kernel ran out
    return X, info


@pytest.mark.parametrize("batch", [1, 5, 37])
def test_push_matches_oracle_on_range_boundaries(batch):
    torch = _torch()
    x_np, _ = signals.batch_r32(batch=batch, N=N, alpha=ALPHA, seed=21 + batch)
    x = torch.from_numpy(x_np).cuda()
    X, info = run(torch, x, 2)
    assert info.staged == 2 and info.cluster == 8 and info.residues == 8
    bins = boundary_bins()
    sigs = sorted({0, batch // 2, batch - 1})
    got = X[torch.tensor(sigs, device="cuda")][:, torch.from_numpy(bins).cuda()].cpu().numpy()
    ref = oracle.alpha_dft(x_np[sigs].astype(np.float64), M, bins=bins)
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= TOL, err
    # no bin of any signal is left unwritten (the output started as NaN in no case: check finiteness)
    assert torch.isfinite(X.view(torch.float32)).all().item()


@pytest.mark.parametrize("batch", [3, 37, 4096])
def test_push_matches_pull_every_bin(batch):
    torch = _torch()
    x_np, _ = signals.batch_r32(batch=batch, N=N, alpha=ALPHA, seed=2)
    x = torch.from_numpy(x_np).cuda()
    Xp, _ = run(torch, x, 2)
    Xl, info = run(torch, x, 0)
    assert info.staged == 0
    num = torch.linalg.vector_norm(Xp - Xl, dim=1)
    den = torch.linalg.vector_norm(Xl, dim=1)
    # same FFT arithmetic, same unpacking formula: agreement far inside the oracle tolerance
    assert (num / den).max().item() <= 1e-6
    del Xp, Xl
    torch.cuda.empty_cache()


def test_push_full_size_first_middle_last_signal_blocks():
    """The benchmark workload (4096 signals) in its launch configuration, against the oracle on
    the range-boundary blocks of the first, middle and last signal of the persistent grid."""
    torch = _torch()
    B = 4096
    x_np, _ = signals.batch_r32(batch=B, N=N, alpha=ALPHA, seed=2)
    x = torch.from_numpy(x_np).cuda()
    X, info = run(torch, x, 2)
    bins = boundary_bins()
    sigs = [0, B // 2, B - 1]
    got = X[torch.tensor(sigs, device="cuda")][:, torch.from_numpy(bins).cuda()].cpu().numpy()
    ref = oracle.alpha_dft(x_np[sigs].astype(np.float64), M, bins=bins)
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= TOL, err
