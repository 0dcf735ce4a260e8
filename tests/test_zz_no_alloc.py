"""adfft_execute_noalloc: the forward transform for callers that cannot allocate
device memory (graph capture, memory owned by another allocator, latency-critical
loops), checked through the C ABI against the plan-based adfft_execute.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2403_16665_gb300 import adfft

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    adfft.load()
    return torch


def _reference(torch, x, M, code):
    B, N = x.shape
    plan = adfft.Plan(N, batch=B, dtype=code, M=M)
    X = torch.empty((B, M), dtype=torch.complex64, device=x.device)
    plan.execute(x.data_ptr(), X.data_ptr())
    torch.cuda.synchronize()
    return X


@pytest.mark.parametrize("code,N,M,batch", [(adfft.R32, 1 << 16, 1 << 19, 4),
                                            (adfft.C64, 1 << 15, 81920, 3),
                                            (adfft.R32, 4096, 32768, 16)])
def test_noalloc_matches_plan_path_twice(code, N, M, batch):
    torch = _torch()
    tol = 2e-6 * np.log2(M)
    rng = np.random.default_rng(N + M)
    for call in range(2):   # two calls in a row share the static scratch
        if code == adfft.R32:
            x_np = rng.standard_normal((batch, N)).astype(np.float32)
        else:
            x_np = (rng.standard_normal((batch, N)) + 1j * rng.standard_normal((batch, N))).astype(np.complex64)
        x = torch.from_numpy(x_np).cuda()
        X = torch.empty((batch, M), dtype=torch.complex64, device="cuda")
        adfft.execute_noalloc(N, M, batch, code, x.data_ptr(), X.data_ptr())
        torch.cuda.synchronize()
        ref = _reference(torch, x, M, code)
        err = (torch.linalg.vector_norm(X - ref, dim=1) / torch.linalg.vector_norm(ref, dim=1)).max().item()
        assert err <= tol, (call, err)


# Small transforms with many residues per column (alpha 2.5, 16, 64): pass-1 shapes with
# a sub-FFT of 2..8 points and up to 64 residues, which only this entry point's geometry
# search reaches; and a shape whose pass 1 needs a cluster of 4 CTAs.  Each is compared
# with the plan path and with the FP64 oracle.
@pytest.mark.parametrize("code,N,M,batch", [(adfft.R32, 8, 512, 3), (adfft.R32, 64, 4096, 2),
                                            (adfft.R32, 16, 40, 5), (adfft.R32, 32, 512, 4),
                                            (adfft.C64, 16, 1024, 3), (adfft.C64, 32, 80, 2),
                                            (adfft.C64, 64, 4096, 2), (adfft.R32, 1 << 17, 1 << 20, 2)])
def test_noalloc_small_and_clustered_shapes(code, N, M, batch):
    torch = _torch()
    import oracle
    tol = 2e-6 * np.log2(M)
    rng = np.random.default_rng(7 * N + M)
    for call in range(2):
        if code == adfft.R32:
            x_np = rng.standard_normal((batch, N)).astype(np.float32)
        else:
            x_np = (rng.standard_normal((batch, N)) + 1j * rng.standard_normal((batch, N))).astype(np.complex64)
        x = torch.from_numpy(x_np).cuda()
        X = torch.full((batch, M), float("nan"), dtype=torch.complex64, device="cuda")
        adfft.execute_noalloc(N, M, batch, code, x.data_ptr(), X.data_ptr())
        torch.cuda.synchronize()
        ref = _reference(torch, x, M, code)
        err = (torch.linalg.vector_norm(X - ref, dim=1) / torch.linalg.vector_norm(ref, dim=1)).max().item()
        assert err <= tol, (call, err)
        if N <= 64:
            got = X.cpu().numpy()
            want = oracle.alpha_dft(x_np.astype(np.complex128 if code == adfft.C64 else np.float64), M)
            e2 = (np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)).max()
            assert e2 <= tol, (call, e2)


def test_noalloc_rejects_what_it_cannot_hold():
    torch = _torch()
    x = torch.zeros(16, device="cuda")
    X = torch.zeros(64, dtype=torch.complex64, device="cuda")
    lib = adfft.load()
    # beyond the 32 MiB scratch: 64 signals x 2^19 complex64 bins
    assert lib.adfft_execute_noalloc(1 << 17, 1 << 20, 64, adfft.R32, x.data_ptr(), X.data_ptr(), None) == -3
    # fp64 inputs are not served by this entry point
    assert lib.adfft_execute_noalloc(16, 64, 1, adfft.R64, x.data_ptr(), X.data_ptr(), None) == -9
    # odd sizes for real input
    assert lib.adfft_execute_noalloc(15, 60, 1, adfft.R32, x.data_ptr(), X.data_ptr(), None) == -3
