"""GPU parity of the two-pass (four-step) form, used when no single-pass shape
fits one cluster's shared memory and selectable by hand otherwise, against the
FP64 oracle on sampled bins."""
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


def tol_for(M, dbl):
    return 1e-12 if dbl else 2e-6 * max(1.0, np.log2(M))


NP = {adfft.R32: np.float32, adfft.R64: np.float64, adfft.C64: np.complex64, adfft.C128: np.complex128}


def run(torch, x, M, code, four_step=False):
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    B, N = xt.shape
    plan = adfft.Plan(N, batch=B, dtype=code, M=M)
    if four_step:
        plan.set_algorithm(adfft.ALGO_FOUR_STEP)
    dbl = code in (adfft.R64, adfft.C128)
    X = torch.empty((B, M), dtype=torch.complex128 if dbl else torch.complex64, device=dev)
    plan.execute(xt.data_ptr(), X.data_ptr())
    plan.sync_status()
    return X, plan


def expected_passes(code, N, M):
    """1 if the default rule finds a single-pass shape: a power-of-two sub-FFT
    length Np dividing gcd(Mc, Nc) (the largest with a fold q <= 64, smaller
    ones with q <= 16) whose P = Mc/Np residues spread over a cluster of at
    most 16 CTAs of 16384 (fp64: 8192) values each; else 2."""
    real = code in (adfft.R32, adfft.R64)
    Nc, Mc = (N // 2, M // 2) if real else (N, M)
    vals = 8192 if code in (adfft.R64, adfft.C128) else 16384
    g = int(np.gcd(Nc, Mc))
    np0 = g & -g
    n = np0
    while n >= 1:
        q, P = Nc // n, Mc // n
        if q > (64 if n == np0 else 16):
            break
        if any(P % c == 0 and (P // c) * n <= vals and P <= 512 for c in range(1, min(16, P) + 1)):
            return 1
        n //= 2
    return 2


def sample_bins(M, n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([np.arange(8), M - 1 - np.arange(8), [M // 2 - 1, M // 2, M // 2 + 1],
                                     rng.integers(0, M, n)]))


@pytest.mark.parametrize("four_step", [False, True])
@pytest.mark.parametrize("code", [adfft.R32, adfft.C64, adfft.R64, adfft.C128])
@pytest.mark.parametrize("N,alpha", [(1 << 15, 2), (1 << 16, 4), (1 << 17, 8), (1 << 16, 2.5),
                                     (1 << 18, 16), (1 << 15, 3)])
def test_two_pass_sampled(code, N, alpha, four_step):
    torch = _torch()
    M = int(round(alpha * N))
    rng = np.random.default_rng(N + M)
    x = rng.standard_normal((2, N))
    if code in (adfft.C64, adfft.C128):
        x = x + 1j * rng.standard_normal((2, N))
    x = x.astype(NP[code])
    X, plan = run(torch, x, M, code, four_step)
    expect = 2 if four_step else expected_passes(code, N, M)
    assert plan.info.passes == expect, (plan.info.passes, plan.info.fft_len)
    assert (plan.workspace_bytes() > 0) == (expect == 2)
    assert plan.info.algo == (adfft.ALGO_FOUR_STEP if expect == 2 else adfft.ALGO_FOLD)
    bins = sample_bins(M, 600, N)
    got = X[:, torch.from_numpy(bins).cuda()].cpu().numpy()
    ref = oracle.alpha_dft(x.astype(np.complex128), M, bins=bins)
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= tol_for(M, code in (adfft.R64, adfft.C128)), err.max()
    if code in (adfft.R32, adfft.R64):
        Xs = X[0].cpu().numpy()
        m = np.arange(1, M)
        assert np.max(np.abs(Xs[M - m] - np.conj(Xs[m]))) <= 1e-5 * np.max(np.abs(Xs))


def test_large_real_workload_sampled():
    """8 real fp32 signals, N = 2^22, alpha = 16 (2^26 bins each): 2 signals on
    sampled bins, including windows around the strongest tones."""
    torch = _torch()
    x, prm = signals.large_r32()
    N, M = 1 << 22, 1 << 26
    X, plan = run(torch, x, M, adfft.R32)
    assert plan.info.passes == 2
    for s in (0, 7):
        top = np.argsort(prm["A"][s])[-3:]
        centers = np.round(prm["nu"][s, top] * 16).astype(np.int64)
        win = (centers[:, None] + np.arange(-8, 9)[None, :]).ravel() % M
        bins = np.unique(np.concatenate([win, sample_bins(M, 160, s)]))
        got = X[s, torch.from_numpy(bins).cuda()].cpu().numpy()
        ref = oracle.alpha_dft(x[s].astype(np.float64), M, bins=bins)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= tol_for(M, False), err


@pytest.mark.parametrize("code,N,alpha", [(adfft.C128, 1 << 14, 2), (adfft.R64, 1 << 15, 2),
                                          (adfft.C128, 1 << 14, 4)])
def test_two_pass_adjoint_matches_oracle(code, N, alpha):
    torch = _torch()
    M = int(round(alpha * N))
    real = code == adfft.R64
    rng = np.random.default_rng(N + 7)
    g = (rng.standard_normal((1, M)) + 1j * rng.standard_normal((1, M)))
    dev = torch.device("cuda:0")
    plan = adfft.Plan(N, batch=1, dtype=code, M=M)
    plan.set_algorithm(adfft.ALGO_FOUR_STEP)
    assert plan.info.passes == 2
    gt = torch.from_numpy(g).to(dev)
    xb = torch.empty((1, N), dtype=torch.float64 if real else torch.complex128, device=dev)
    plan.execute_adjoint(gt.data_ptr(), xb.data_ptr())
    plan.sync_status()
    ref = oracle.alpha_dft_adjoint(g, N, real_input=real)
    got = xb.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12


@pytest.mark.parametrize("four_step", [False, True])
@pytest.mark.parametrize("code,N,alpha", [(adfft.R32, 1 << 17, 8), (adfft.C64, 1 << 15, 3),
                                          (adfft.R32, 1 << 17, 2.5), (adfft.R32, 1 << 22, 16)])
def test_two_pass_adjoint_dot_product(code, N, alpha, four_step):
    """<A x, g> = <x, A^H g> through the forward and adjoint two-pass launches."""
    torch = _torch()
    M = int(round(alpha * N))
    real = code == adfft.R32
    dev = torch.device("cuda:0")
    gen = torch.Generator(device=dev).manual_seed(5)
    if real:
        x = torch.randn((1, N), device=dev, generator=gen)
    else:
        x = torch.randn((1, N), device=dev, generator=gen, dtype=torch.complex64)
    g = torch.randn((1, M), device=dev, generator=gen, dtype=torch.complex64)
    plan = adfft.Plan(N, batch=1, dtype=code, M=M)
    if four_step:
        plan.set_algorithm(adfft.ALGO_FOUR_STEP)
    assert plan.info.passes == (2 if four_step else expected_passes(code, N, M))
    X = torch.empty((1, M), dtype=torch.complex64, device=dev)
    xb = torch.empty_like(x)
    plan.execute(x.data_ptr(), X.data_ptr())
    plan.execute_adjoint(g.data_ptr(), xb.data_ptr())
    plan.sync_status()
    lhs = torch.vdot(g.flatten().to(torch.complex128), X.flatten().to(torch.complex128))
    rhs = torch.vdot(xb.flatten().to(torch.complex128), x.flatten().to(torch.complex128))
    if real:
        lhs, rhs = lhs.real, rhs.real
    assert abs((lhs - rhs).item()) <= 5e-6 * max(1.0, abs(lhs.item())) * np.sqrt(np.log2(M))


@pytest.mark.parametrize("code,N,alpha,batch", [(adfft.R32, 1 << 22, 16, 2), (adfft.R32, 1 << 17, 8, 3),
                                                (adfft.C64, 1 << 16, 16, 2)])
def test_two_pass_fp32_adjoint_elementwise(code, N, alpha, batch):
    """FP32 two-pass adjoint element by element against the oracle's explicit adjoint, at
    sampled output samples (first, last, column and block boundaries of the four-step split,
    random) of every signal, including the 2^22-sample, alpha = 16 workload."""
    torch = _torch()
    M = int(round(alpha * N))
    real = code == adfft.R32
    rng = np.random.default_rng(N + batch)
    g = (rng.standard_normal((batch, M)) + 1j * rng.standard_normal((batch, M))).astype(np.complex64)
    dev = torch.device("cuda:0")
    plan = adfft.Plan(N, batch=batch, dtype=code, M=M)
    plan.set_algorithm(adfft.ALGO_FOUR_STEP)
    info = plan.info
    assert info.passes == 2
    gt = torch.from_numpy(g).to(dev)
    xb = torch.empty((batch, N), dtype=torch.float32 if real else torch.complex64, device=dev)
    plan.execute_adjoint(gt.data_ptr(), xb.data_ptr())
    plan.sync_status()
    A = info.four_step_a
    edges = [0, 1, N - 1, N // 2, A - 1, A, N - A, 2 * A + 1]
    samples = np.unique(np.concatenate([np.array(edges) % N, rng.integers(0, N, 24)]))
    got = xb[:, torch.from_numpy(samples).to(dev)].cpu().numpy()
    ref = oracle.alpha_dft_adjoint(g.astype(np.complex128), N, real_input=real, samples=samples)
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= tol_for(M, False), err
