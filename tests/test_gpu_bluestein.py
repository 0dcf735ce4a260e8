"""GPU parity of the chirp-z (Bluestein) path against the FP64 oracle: sizes the
fold path cannot take (gcd(M, N) not a power of two), and the complex64
N = 8192, alpha in {2.5, 3.75} workload forced onto the chirp-z kernel."""
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


def run(torch, x, M, dtype_code, algo=None):
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    B, N = xt.shape
    plan = adfft.Plan(N, batch=B, dtype=dtype_code, M=M)
    if algo is not None:
        plan.set_algorithm(algo)
    dbl = dtype_code in (adfft.R64, adfft.C128)
    X = torch.empty((B, M), dtype=torch.complex128 if dbl else torch.complex64, device=dev)
    plan.execute(xt.data_ptr(), X.data_ptr())
    torch.cuda.synchronize()
    return X.cpu().numpy(), plan


NP = {adfft.R32: np.float32, adfft.R64: np.float64, adfft.C64: np.complex64, adfft.C128: np.complex128}


@pytest.mark.parametrize("dtype_code", [adfft.R32, adfft.C64, adfft.R64, adfft.C128])
@pytest.mark.parametrize("N,M", [(7, 7), (9, 6), (3, 10), (100, 250), (1000, 2000), (1000, 2500),
                                 (1000, 300), (999, 3996), (3000, 7500), (5000, 12345)])
def test_chirp_z_sizes(dtype_code, N, M):
    torch = _torch()
    dbl = dtype_code in (adfft.R64, adfft.C128)
    if dbl and 2 * N > 8192:
        # the FP64 chirp-z kernel holds a padded length of at most 8192 in one CTA; a refusal
        # of the forced algorithm is that stated limit
        try:
            adfft.Plan(N, batch=1, dtype=dtype_code, M=M).set_algorithm(adfft.ALGO_BLUESTEIN)
        except adfft.AdfftError as e:
            if e.code not in (-3, -9):
                raise
            pytest.skip("fp64 chirp-z beyond a padded length of 8192 (2N - 1 > 8192): %s" % e)
    rng = np.random.default_rng(N * 13 + M)
    x = rng.standard_normal((2, N))
    if dtype_code in (adfft.C64, adfft.C128):
        x = x + 1j * rng.standard_normal((2, N))
    x = x.astype(NP[dtype_code])
    got, plan = run(torch, x, M, dtype_code, algo=adfft.ALGO_BLUESTEIN)
    assert plan.info.algo == adfft.ALGO_BLUESTEIN
    ref = oracle.alpha_dft(x.astype(np.complex128), M)
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= tol_for(M, dbl), (err.max(), plan.info.fft_len, plan.info.residues)


@pytest.mark.parametrize("alpha", [2.5, 3.75])
def test_complex_workload_forced_chirp_z(alpha):
    """1024-signal complex64 workload shape (8 signals here), N = 8192, on the
    chirp-z kernel; sampled bins against the oracle and all bins against the fold path."""
    torch = _torch()
    x, _ = signals.batch_c64(batch=8, alpha=alpha)
    M = int(round(alpha * 8192))
    got, plan = run(torch, x, M, adfft.C64, algo=adfft.ALGO_BLUESTEIN)
    assert plan.info.algo == adfft.ALGO_BLUESTEIN
    rng = np.random.default_rng(5)
    bins = np.unique(np.concatenate([np.arange(16), M - 1 - np.arange(16), rng.integers(0, M, 2000)]))
    ref = oracle.alpha_dft(x.astype(np.complex128), M, bins=bins)
    err = np.linalg.norm(got[:, bins] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= tol_for(M, False)
    fold, _ = run(torch, x, M, adfft.C64, algo=adfft.ALGO_FOLD)
    d = np.linalg.norm(got - fold, axis=1) / np.linalg.norm(fold, axis=1)
    assert d.max() <= 2 * tol_for(M, False)


@pytest.mark.parametrize("N,M", [(1000, 2000), (1000, 2500), (999, 3996), (300, 750)])
def test_auto_picks_chirp_z_when_no_power_of_two_divisor_gives_a_small_fold(N, M):
    """Every power-of-two divisor g' of gcd(M, N) leaves a fold N/g' > 64 here."""
    _torch()
    for code in (adfft.R32, adfft.C64):
        assert adfft.Plan(N, batch=1, dtype=code, M=M).info.algo == adfft.ALGO_BLUESTEIN


def test_single_real_fp64_chirp_z():
    torch = _torch()
    x, _ = signals.single_r64()
    got, _ = run(torch, x, 4096, adfft.R64, algo=adfft.ALGO_BLUESTEIN)
    ref = oracle.alpha_dft(x, 4096)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12


@pytest.mark.parametrize("code,N,M,batch,force", [
    (adfft.C64, 1000, 2500, 2, False),       # chirp-z only (no power-of-two common divisor): one tile
    (adfft.R32, 1000, 2500, 3, False),
    (adfft.C128, 300, 700, 2, False),
    (adfft.R64, 1000, 2500, 2, False),
    (adfft.C64, 8192, 20480, 2, True),       # forced chirp-z: N + M - 1 > L, input in 3 blocks
    (adfft.C64, 1024, 100000, 1, True),      # 13 input blocks
    (adfft.R32, 6000, 15000, 2, False),      # 2 output chunks x 2 input blocks
    (adfft.C128, 3000, 7500, 1, False),      # fp64: L = 8192, blocks of 4096
])
def test_chirp_z_adjoint_matches_oracle(code, N, M, batch, force):
    """The chirp-z adjoint (correlation of g conj(c) with the chirp, blocked) against the
    oracle's explicit adjoint of Eq. 7 at every output sample."""
    torch = _torch()
    real = code in (adfft.R32, adfft.R64)
    dbl = code in (adfft.R64, adfft.C128)
    rng = np.random.default_rng(N + M)
    g = (rng.standard_normal((batch, M)) + 1j * rng.standard_normal((batch, M))).astype(
        np.complex128 if dbl else np.complex64)
    plan = adfft.Plan(N, batch=batch, dtype=code, M=M)
    if force:
        plan.set_algorithm(adfft.ALGO_BLUESTEIN)
    assert plan.info.algo == adfft.ALGO_BLUESTEIN
    gt = torch.from_numpy(g).cuda()
    xt = torch.float64 if (real and dbl) else torch.float32 if real else torch.complex128 if dbl else torch.complex64
    xb = torch.empty((batch, N), dtype=xt, device="cuda")
    plan.execute_adjoint(gt.data_ptr(), xb.data_ptr())
    plan.sync_status()
    ref = oracle.alpha_dft_adjoint(g.astype(np.complex128), N, real_input=real)
    got = xb.cpu().numpy()
    err = (np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)).max()
    assert err <= (1e-12 if dbl else 2e-6 * np.log2(M)), err


def test_chirp_z_adjoint_dot_product():
    """<A x, g> = <x, A^H g> through the chirp-z forward and adjoint launches."""
    torch = _torch()
    N, M = 1000, 2500
    x = torch.randn((2, N), dtype=torch.complex128, device="cuda")
    g = torch.randn((2, M), dtype=torch.complex128, device="cuda")
    plan = adfft.Plan(N, batch=2, dtype=adfft.C128, M=M)
    X = torch.empty((2, M), dtype=torch.complex128, device="cuda")
    xb = torch.empty_like(x)
    plan.execute(x.data_ptr(), X.data_ptr())
    plan.execute_adjoint(g.data_ptr(), xb.data_ptr())
    plan.sync_status()
    lhs = torch.vdot(g.flatten(), X.flatten())
    rhs = torch.vdot(xb.flatten(), x.flatten())
    assert abs((lhs - rhs).item()) <= 1e-11 * abs(lhs.item())
