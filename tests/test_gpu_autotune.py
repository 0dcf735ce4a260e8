"""GPU parity of the fold form's launch shapes (sub-FFT lengths below gcd(M, N),
cluster sizes, input staging, the two-pass alternative) and of the autotuner that
chooses among them, against the FP64 oracle and against each other."""
import json

import numpy as np
import pytest

import oracle
from paper_2403_16665_gb300 import adfft, signals

pytestmark = pytest.mark.gpu

NP = {adfft.R32: np.float32, adfft.R64: np.float64, adfft.C64: np.complex64, adfft.C128: np.complex128}


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    adfft.load()
    return torch


def tol_for(M, dbl):
    return 1e-12 if dbl else 2e-6 * max(1.0, np.log2(M))


def sample_bins(M, n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([np.arange(8), M - 1 - np.arange(8), [M // 2 - 1, M // 2, M // 2 + 1],
                                     rng.integers(0, M, n)]))


def make_input(code, B, N, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, N))
    if code in (adfft.C64, adfft.C128):
        x = x + 1j * rng.standard_normal((B, N))
    return x.astype(NP[code])


def forward(torch, plan, xt, M, dbl):
    X = torch.empty((xt.shape[0], M), dtype=torch.complex128 if dbl else torch.complex64, device=xt.device)
    plan.execute(xt.data_ptr(), X.data_ptr())
    plan.sync_status()
    return X


def adjoint(torch, plan, g, N, in_dtype):
    xb = torch.empty((g.shape[0], N), dtype=in_dtype, device=g.device)
    plan.execute_adjoint(g.data_ptr(), xb.data_ptr())
    plan.sync_status()
    return xb


def rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return (np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)).max()


# sub-FFT beyond one CTA: the default rule halves the sub-FFT length (fold of 2
# blocks) and stays single-pass; the two-pass form is the forced alternative
@pytest.mark.parametrize("code,N,alpha,fft_len,cluster", [
    (adfft.R32, 1 << 16, 2, 16384, 4), (adfft.R32, 1 << 16, 3, 16384, 6), (adfft.R32, 1 << 16, 4, 16384, 8),
    (adfft.R32, 1 << 16, 8, 16384, 16), (adfft.C64, 1 << 15, 2, 16384, 4), (adfft.R64, 1 << 15, 4, 8192, 8),
    (adfft.R32, 1 << 16, 2.5, 16384, 5), (adfft.R32, 1 << 15, 8, 16384, 8), (adfft.R32, 1 << 15, 3, 16384, 3),
])
def test_halved_sub_fft_single_pass(code, N, alpha, fft_len, cluster):
    torch = _torch()
    dbl = code in (adfft.R64, adfft.C128)
    real = code in (adfft.R32, adfft.R64)
    M = int(round(alpha * N))
    x = make_input(code, 2, N, N + M)
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(x).to(dev)
    plan = adfft.Plan(N, batch=2, dtype=code, M=M)
    info = plan.info
    assert (info.algo, info.passes, info.fft_len, info.cluster) == (adfft.ALGO_FOLD, 1, fft_len, cluster)
    assert info.fold == (N // 2 if real else N) // fft_len
    assert plan.workspace_bytes() == 0
    X = forward(torch, plan, xt, M, dbl)
    bins = sample_bins(M, 800, N)
    got = X[:, torch.from_numpy(bins).to(dev)].cpu().numpy()
    ref = oracle.alpha_dft(x.astype(np.complex128), M, bins=bins)
    assert rel(got, ref) <= tol_for(M, dbl)
    if real:
        Xs = X[0].cpu().numpy()
        m = np.arange(1, M)
        assert np.max(np.abs(Xs[M - m] - np.conj(Xs[m]))) <= (1e-12 if dbl else 1e-5) * np.max(np.abs(Xs))
    # the two-pass form on the same plan, and the adjoints of both forms
    g = torch.randn((2, M), dtype=torch.complex128 if dbl else torch.complex64, device=dev)
    xb1 = adjoint(torch, plan, g, N, xt.dtype).cpu().numpy()
    plan.set_algorithm(adfft.ALGO_FOUR_STEP)
    assert plan.info.passes == 2 and plan.workspace_bytes() > 0
    X2 = forward(torch, plan, xt, M, dbl)
    assert rel(X.cpu().numpy(), X2.cpu().numpy()) <= 2 * tol_for(M, dbl)
    xb2 = adjoint(torch, plan, g, N, xt.dtype).cpu().numpy()
    assert rel(xb1, xb2) <= 2 * tol_for(M, dbl)
    # <A x, g> = <x, A^H g> (real inputs: the real part)
    lhs = np.vdot(X.cpu().numpy().astype(np.complex128), g.cpu().numpy().astype(np.complex128))
    rhs = np.vdot(x.astype(np.complex128), xb1.astype(np.complex128))
    if real:
        lhs, rhs = lhs.real, rhs.real
    scale = np.linalg.norm(X.cpu().numpy()) * np.linalg.norm(g.cpu().numpy())
    assert abs(lhs - rhs) <= 10 * tol_for(M, dbl) * scale
    plan.set_algorithm(adfft.ALGO_AUTO)
    assert plan.info.passes == 1


# gcd(M, N) not a power of two, but with a power-of-two divisor that leaves a small fold
@pytest.mark.parametrize("code,N,M", [(adfft.C64, 12288, 24576), (adfft.R32, 6144, 18432),
                                      (adfft.C128, 3 * 1024, 5 * 1024), (adfft.R32, 5 * 2048, 7 * 2048),
                                      (adfft.R32, 100, 250), (adfft.C64, 100, 250), (adfft.R64, 100, 250)])
def test_fold_with_non_power_of_two_gcd(code, N, M):
    torch = _torch()
    dbl = code in (adfft.R64, adfft.C128)
    real = code in (adfft.R32, adfft.R64)
    x = make_input(code, 2, N, N * 7 + M)
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(x).to(dev)
    plan = adfft.Plan(N, batch=2, dtype=code, M=M)
    assert plan.info.algo == adfft.ALGO_FOLD and plan.info.fold > 1
    X = forward(torch, plan, xt, M, dbl)
    bins = sample_bins(M, 1500, M)
    got = X[:, torch.from_numpy(bins).to(dev)].cpu().numpy()
    ref = oracle.alpha_dft(x.astype(np.complex128), M, bins=bins)
    assert rel(got, ref) <= tol_for(M, dbl), (plan.info.fft_len, plan.info.fold)
    g = np.random.default_rng(M).standard_normal((2, M)) + 1j * np.random.default_rng(N).standard_normal((2, M))
    g = g.astype(np.complex128 if dbl else np.complex64)
    xb = adjoint(torch, plan, torch.from_numpy(g).to(dev), N, xt.dtype).cpu().numpy()
    ref_b = oracle.alpha_dft_adjoint(g[:1].astype(np.complex128), N, real_input=real)
    assert rel(xb[:1], ref_b) <= tol_for(M, dbl)


def candidate_shapes(code, N, M):
    """The fold shapes the autotuner tries (sub-FFT length, cluster, staging)."""
    real = code in (adfft.R32, adfft.R64)
    dbl = code in (adfft.R64, adfft.C128)
    Nc, Mc = (N // 2, M // 2) if real else (N, M)
    g = int(np.gcd(Nc, Mc))
    np0 = g & -g
    vals = (16 if dbl else 32) * 512
    out = []
    np_ = np0
    while np_ >= 1:
        if np_ != np0 and (Nc // np_ > 16 or np_ < 64):
            break
        P = Mc // np_
        for c in range(1, min(16, P) + 1):
            if P % c == 0 and (P // c) * np_ <= vals:
                out += [(np_, c, 1), (np_, c, 0)]
        np_ //= 2
    return out


@pytest.mark.parametrize("code,N,alpha", [(adfft.R32, 4096, 8), (adfft.C64, 2048, 2.5), (adfft.R64, 1024, 4),
                                          (adfft.C64, 1024, 16)])
def test_every_candidate_shape_matches_the_oracle(code, N, alpha):
    torch = _torch()
    dbl = code in (adfft.R64, adfft.C128)
    real = code in (adfft.R32, adfft.R64)
    M = int(round(alpha * N))
    B = 3
    x = make_input(code, B, N, N + 11 * M)
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(x).to(dev)
    ref = oracle.alpha_dft(x.astype(np.complex128), M)
    g = np.random.default_rng(5 * M).standard_normal((B, M)) + 1j * np.random.default_rng(N).standard_normal((B, M))
    g = g.astype(np.complex128 if dbl else np.complex64)
    gt = torch.from_numpy(g).to(dev)
    ref_b = oracle.alpha_dft_adjoint(g.astype(np.complex128), N, real_input=real)
    plan = adfft.Plan(N, batch=B, dtype=code, M=M)
    ran = 0
    for fft_len, cluster, staged in candidate_shapes(code, N, M):
        for grid in (0, 1):   # resident-size grid (here one cluster per signal), and one cluster for all
            try:
                plan.set_launch_shape(fft_len, cluster, staged, grid)
            except adfft.AdfftError as e:
                assert e.code == -9, (fft_len, cluster, staged, e)   # does not fit: NOT_SUPPORTED
                continue
            info = plan.info
            assert (info.fft_len, info.cluster, info.staged) == (fft_len, cluster, staged)
            assert info.grid == (1 if grid == 1 else B)
            X = forward(torch, plan, xt, M, dbl).cpu().numpy()
            assert rel(X, ref) <= tol_for(M, dbl), (fft_len, cluster, staged, grid)
            xb = adjoint(torch, plan, gt, N, xt.dtype).cpu().numpy()
            assert rel(xb, ref_b) <= tol_for(M, dbl), (fft_len, cluster, staged, grid)
            ran += 1
    assert ran >= 8


@pytest.mark.parametrize("staged", [1, 0])
def test_grid_size_does_not_change_results(staged):
    """Clusters loop over signals (persistent grid); every signal is transformed by
    the same arithmetic whichever cluster takes it, so all grids agree bit for bit."""
    torch = _torch()
    B, N, M = 100, 16384, 131072
    x, _ = signals.batch_r32(batch=B)
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(x).to(dev)
    plan = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    g = torch.randn((B, M), dtype=torch.complex64, device=dev)
    outs, grads = [], []
    for grid in (-1, 0, 1, 7):
        plan.set_launch_shape(8192, 4, staged, grid)
        assert plan.info.grid == {-1: B, 1: 1, 7: 7}.get(grid, plan.info.grid)
        if grid == 0:
            assert 1 <= plan.info.grid <= B
        outs.append(forward(torch, plan, xt, M, False))
        grads.append(adjoint(torch, plan, g, N, xt.dtype))
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    for o in grads[1:]:
        assert torch.equal(o, grads[0])
    sig = np.array([0, 37, 99])
    bins = sample_bins(M, 400, 3)
    got = outs[0][torch.from_numpy(sig).to(dev)][:, torch.from_numpy(bins).to(dev)].cpu().numpy()
    ref = oracle.alpha_dft(x[sig].astype(np.float64), M, bins=bins)
    assert rel(got, ref) <= tol_for(M, False)


def test_autotune_forward_and_cache(tmp_path):
    torch = _torch()
    adfft.autotune_clear()
    B, N, alpha = 64, 16384, 8
    M = N * alpha
    x, _ = signals.batch_r32(batch=B)
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(x).to(dev)
    plan = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    assert plan.info.tuned == 0
    X0 = forward(torch, plan, xt, M, False).cpu().numpy()
    X = torch.empty((B, M), dtype=torch.complex64, device=dev)
    plan.autotune(xt.data_ptr(), X.data_ptr(), iters=2)
    info = plan.info
    assert info.tuned == 1 and info.algo in (adfft.ALGO_FOLD, adfft.ALGO_FOUR_STEP)
    X1 = forward(torch, plan, xt, M, False).cpu().numpy()
    assert rel(X1, X0) <= 2 * tol_for(M, False)
    # a new plan of the same sizes takes the cached shape; a different batch does not
    p2 = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    assert p2.info.tuned == 1
    assert (p2.info.algo, p2.info.fft_len, p2.info.cluster, p2.info.staged) == \
        (info.algo, info.fft_len, info.cluster, info.staged)
    assert adfft.Plan(N, batch=B + 1, dtype=adfft.R32, M=M).info.tuned == 0
    path = tmp_path / "tune.json"
    adfft.autotune_save(str(path))
    entries = json.loads(path.read_text())["entries"]
    assert len(entries) == 1 and entries[0]["N"] == N and entries[0]["batch"] == B
    adfft.autotune_clear()
    assert adfft.Plan(N, batch=B, dtype=adfft.R32, M=M).info.tuned == 0
    adfft.autotune_load(str(path))
    p3 = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    assert p3.info.tuned == 1 and p3.info.fft_len == info.fft_len
    X3 = forward(torch, p3, xt, M, False).cpu().numpy()
    assert rel(X3, X1) <= 1e-7
    # entries of another GPU are kept but never applied
    e = dict(entries[0], device="some other GPU|sm_90|cuda-driver 1", N=8192, M=65536)
    path.write_text(json.dumps({"adfft_autotune": 1, "entries": [e]}))
    adfft.autotune_load(str(path))
    assert adfft.Plan(8192, batch=B, dtype=adfft.R32, M=65536).info.tuned == 0
    adfft.autotune_clear()


def test_autotune_ragged():
    torch = _torch()
    adfft.autotune_clear()
    Ns, alphas = signals.ragged_shapes(count=120, seed=9)
    plan = adfft.RaggedPlan(Ns, alphas)
    dev = torch.device("cuda:0")
    x = torch.randn(int(plan.in_off[-1]), device=dev)
    X0 = torch.empty(int(plan.out_off[-1]), dtype=torch.complex64, device=dev)
    plan.execute(x.data_ptr(), X0.data_ptr())
    X = torch.empty_like(X0)
    plan.autotune(x.data_ptr(), X.data_ptr(), iters=1, with_adjoint=True)   # forward + backward steps
    assert plan.info.tuned == 1
    X1 = torch.empty_like(X0)
    plan.execute(x.data_ptr(), X1.data_ptr())   # captures a new graph with the tuned shapes
    g = torch.randn_like(X0)
    xb = torch.empty_like(x)
    plan.execute_adjoint(g.data_ptr(), xb.data_ptr())
    plan.sync_status()
    for i in range(len(Ns)):
        N, M = int(Ns[i]), int(round(alphas[i] * Ns[i]))
        a, b = X1[plan.out_off[i]:plan.out_off[i + 1]], X0[plan.out_off[i]:plan.out_off[i + 1]]
        assert (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item() <= 2 * tol_for(M, False), (i, N, M)
        p = adfft.Plan(N, batch=1, dtype=adfft.R32, M=M)   # a uniform plan of the same sizes
        gi = g[plan.out_off[i]:plan.out_off[i + 1]].contiguous()
        xbi = torch.empty(N, device=dev)
        p.execute_adjoint(gi.data_ptr(), xbi.data_ptr())
        torch.cuda.synchronize()
        ref = xbi
        got = xb[plan.in_off[i]:plan.in_off[i + 1]]
        assert (torch.linalg.norm(got - ref) / torch.linalg.norm(ref)).item() <= 2 * tol_for(M, False), (i, N, M)
    adfft.autotune_clear()


@pytest.mark.parametrize("N,alpha,B", [(16384, 8, 6), (32768, 4, 3), (16384, 8, 45)])
@pytest.mark.parametrize("cluster,staged", [(4, 1), (4, 0), (8, 1), (8, 0)])
def test_specialised_sub_fft_8192_shapes(N, alpha, B, cluster, staged):
    """Real fp32 plans whose packed sub-FFT is 8192 points with 8 residues run
    compile-time specialised kernels (clusters of 4 with 2 residues per CTA, or of 8
    with 1; N = 32768, alpha = 4: sub-FFT halved, fold of 2).  All bins against the
    generic kernel (sub-FFT 4096), sampled bins against the oracle, every grid size
    bit for bit."""
    torch = _torch()
    M = alpha * N
    x = make_input(adfft.R32, B, N, 17 * N + B)
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(x).to(dev)
    plan = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    plan.set_launch_shape(4096, 4, 0, 0)   # generic kernel: 16 residues of 4096 points
    X_ref = forward(torch, plan, xt, M, False)
    outs = []
    for grid in (0, -1, 1, 2):
        try:
            plan.set_launch_shape(8192, cluster, staged, grid)
        except adfft.AdfftError as e:
            assert e.code == -9 and staged == 1   # the signal does not fit next to the regions
            pytest.skip("staging does not fit this shape")
        info = plan.info
        assert (info.fft_len, info.residues, info.cluster, info.staged) == (8192, 8, cluster, staged)
        outs.append(forward(torch, plan, xt, M, False))
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    X = outs[0].cpu().numpy()
    assert rel(X, X_ref.cpu().numpy()) <= 2 * tol_for(M, False)
    bins = np.unique(np.concatenate([sample_bins(M, 700, N), [M // 4, M // 4 + 1, M // 2, M // 2 + 1,
                                                               3 * M // 4, 3 * M // 4 + 1, M - 2, M - 1]]))
    sig = np.array([0, B - 1])
    ref = oracle.alpha_dft(x[sig].astype(np.float64), M, bins=bins)
    assert rel(X[sig][:, bins], ref) <= tol_for(M, False)
    m = np.arange(1, M)
    assert np.max(np.abs(X[0][M - m] - np.conj(X[0][m]))) <= 1e-5 * np.max(np.abs(X[0]))


def test_autotune_four_step_split():
    """A plan only the four-step form serves (N = 2^18 real, alpha = 16): the autotuner
    times every split Nc = A B; the tuned plan agrees with the default one and with the
    oracle on sampled bins, and the split is recorded in the cache."""
    torch = _torch()
    adfft.autotune_clear()
    B, N, alpha = 2, 1 << 18, 16
    M = N * alpha
    x = make_input(adfft.R32, B, N, 99)
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(x).to(dev)
    plan = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    assert plan.info.passes == 2
    X0 = forward(torch, plan, xt, M, False).cpu().numpy()
    X = torch.empty((B, M), dtype=torch.complex64, device=dev)
    plan.autotune(xt.data_ptr(), X.data_ptr(), iters=1)
    info = plan.info
    assert info.tuned == 1 and info.passes == 2 and info.four_step_a * (info.fft_len // info.four_step_a) == N // 2
    X1 = forward(torch, plan, xt, M, False).cpu().numpy()
    assert rel(X1, X0) <= 2 * tol_for(M, False)
    bins = sample_bins(M, 500, 7)
    ref = oracle.alpha_dft(x.astype(np.float64), M, bins=bins)
    assert rel(X1[:, bins], ref) <= tol_for(M, False)
    p2 = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    assert p2.info.tuned == 1 and p2.info.four_step_a == info.four_step_a
    X2 = forward(torch, p2, xt, M, False).cpu().numpy()
    assert rel(X2, X1) <= 1e-7
    adfft.autotune_clear()
