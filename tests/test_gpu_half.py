"""Half-spectrum output for real input (X_0 .. X_{M/2}; the rest is conj-symmetric,
X_{M-m} = conj X_m, Sec. 2 Eq. 2's negative frequencies): the forward equals the first
M/2 + 1 bins of the full-spectrum plan bit for bit and the FP64 oracle on sampled bins;
the adjoint equals the oracle's adjoint of the gradient extended by zeros above M/2 (real
part); plans without that form refuse it."""
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


def tol(M, dbl):
    return 1e-12 if dbl else 2e-6 * np.log2(M)


CASES = [(adfft.R32, 16384, 8, 5), (adfft.R32, 4096, 8, 3), (adfft.R32, 2048, 2.5, 3), (adfft.R32, 1024, 3, 2),
         (adfft.R32, 65536, 4, 2), (adfft.R32, 256, 2, 7), (adfft.R64, 1024, 4, 2), (adfft.R64, 4096, 8, 2)]


@pytest.mark.parametrize("code,N,alpha,batch", CASES)
def test_half_spectrum_forward(code, N, alpha, batch):
    torch = _torch()
    M = int(round(alpha * N))
    dbl = code == adfft.R64
    rng = np.random.default_rng(N + batch)
    x_np = rng.standard_normal((batch, N)).astype(np.float64 if dbl else np.float32)
    x = torch.from_numpy(x_np).cuda()
    ct = torch.complex128 if dbl else torch.complex64
    full = adfft.Plan(N, batch=batch, dtype=code, M=M)
    Xf = torch.empty((batch, M), dtype=ct, device="cuda")
    full.execute(x.data_ptr(), Xf.data_ptr())
    half = adfft.Plan(N, batch=batch, dtype=code, M=M)
    half.set_output(adfft.OUTPUT_HALF)
    assert half.info.out_bins == M // 2 + 1
    Xh = torch.full((batch, M // 2 + 1), complex(float("nan"), float("nan")), dtype=ct, device="cuda")
    half.execute(x.data_ptr(), Xh.data_ptr())
    half.sync_status()
    assert torch.equal(Xh, Xf[:, : M // 2 + 1])
    bins = np.unique(np.concatenate([[0, 1, M // 2 - 1, M // 2], rng.integers(0, M // 2 + 1, 400)]))
    ref = oracle.alpha_dft(x_np.astype(np.float64), M, bins=bins)
    got = Xh[:, torch.from_numpy(bins).cuda()].cpu().numpy()
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= tol(M, dbl), err


@pytest.mark.parametrize("code,N,alpha,batch", CASES)
def test_half_spectrum_adjoint(code, N, alpha, batch):
    torch = _torch()
    M = int(round(alpha * N))
    H = M // 2 + 1
    dbl = code == adfft.R64
    rng = np.random.default_rng(3 * N + batch)
    g = (rng.standard_normal((batch, H)) + 1j * rng.standard_normal((batch, H))).astype(
        np.complex128 if dbl else np.complex64)
    plan = adfft.Plan(N, batch=batch, dtype=code, M=M)
    plan.set_output(adfft.OUTPUT_HALF)
    gt = torch.from_numpy(g).cuda()
    xb = torch.empty((batch, N), dtype=torch.float64 if dbl else torch.float32, device="cuda")
    plan.execute_adjoint(gt.data_ptr(), xb.data_ptr())
    plan.sync_status()
    g_ext = np.zeros((batch, M), dtype=np.complex128)
    g_ext[:, :H] = g
    if N * M <= (1 << 26):
        ref = oracle.alpha_dft_adjoint(g_ext, N, real_input=True)
        got = xb.cpu().numpy()
    else:
        samples = np.unique(np.concatenate([[0, 1, N - 1], rng.integers(0, N, 48)]))
        ref = oracle.alpha_dft_adjoint(g_ext, N, real_input=True, samples=samples)
        got = xb[:, torch.from_numpy(samples).cuda()].cpu().numpy()
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= tol(M, dbl), err


def test_half_spectrum_dot_product_fp64():
    """<A_h x, g> = <x, A_h^T g> over the reals for the half-spectrum map."""
    torch = _torch()
    N, M = 2048, 5120
    x = torch.randn((2, N), dtype=torch.float64, device="cuda")
    g = torch.randn((2, M // 2 + 1), dtype=torch.complex128, device="cuda")
    plan = adfft.Plan(N, batch=2, dtype=adfft.R64, M=M)
    plan.set_output(adfft.OUTPUT_HALF)
    X = torch.empty((2, M // 2 + 1), dtype=torch.complex128, device="cuda")
    xb = torch.empty_like(x)
    plan.execute(x.data_ptr(), X.data_ptr())
    plan.execute_adjoint(g.data_ptr(), xb.data_ptr())
    plan.sync_status()
    lhs = (torch.conj(g) * X).sum().real.item()
    rhs = (xb * x).sum().item()
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))


def test_half_spectrum_refused_where_unavailable():
    _torch()
    pc = adfft.Plan(1024, batch=1, dtype=adfft.C64, M=4096)          # complex input
    with pytest.raises(adfft.AdfftError):
        pc.set_output(adfft.OUTPUT_HALF)
    po = adfft.Plan(1001, batch=1, dtype=adfft.R32, M=2002)          # odd N: no packed form
    with pytest.raises(adfft.AdfftError):
        po.set_output(adfft.OUTPUT_HALF)
    ph = adfft.Plan(4096, batch=1, dtype=adfft.R32, M=32768)
    ph.set_output(adfft.OUTPUT_HALF)
    with pytest.raises(adfft.AdfftError):
        ph.set_algorithm(adfft.ALGO_FOUR_STEP)
    with pytest.raises(adfft.AdfftError):
        ph.set_launch_shape(2048, 8, 2, 0)                            # the push form: full spectrum only
    ph.set_output(adfft.OUTPUT_FULL)
    assert ph.info.out_bins == 32768
