"""GPU parity of ragged plans (signals of uneven N and alpha packed back to back,
one graph per execute) against uniform plans and the FP64 oracle."""
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


def make_ragged(torch, Ns, alphas, seed=0):
    import ctypes
    lib = adfft.load()
    n = len(Ns)
    Na = np.ascontiguousarray(np.asarray(Ns, dtype=np.int64))
    Aa = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    h = lib.adfft_plan_create_ragged(Na.ctypes.data_as(ctypes.c_void_p), Aa.ctypes.data_as(ctypes.c_void_p),
                                     n, adfft.R32)
    assert h, adfft.STATUS[lib.adfft_last_error()]
    in_off = np.zeros(n + 1, dtype=np.int64)
    out_off = np.zeros(n + 1, dtype=np.int64)
    assert lib.adfft_plan_offsets(h, in_off.ctypes.data_as(ctypes.c_void_p), out_off.ctypes.data_as(ctypes.c_void_p)) == 0
    return lib, ctypes.c_void_p(h), in_off, out_off


def test_ragged_forward_and_adjoint_against_uniform_plans():
    torch = _torch()
    rng = np.random.default_rng(3)
    Ns = [int(2 ** e) for e in rng.integers(8, 17, size=40)] + [65536, 256, 32768]
    alphas = list(rng.choice([2.0, 3.0, 4.0, 8.0, 2.5], size=len(Ns)))
    lib, h, in_off, out_off = make_ragged(torch, Ns, alphas)
    dev = torch.device("cuda:0")
    x = torch.randn(int(in_off[-1]), device=dev)
    X = torch.empty(int(out_off[-1]), dtype=torch.complex64, device=dev)
    s = torch.cuda.current_stream().cuda_stream
    import ctypes
    for _ in range(2):   # the second call replays the captured graph
        assert lib.adfft_execute(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(s)) == 0
    g = torch.randn(int(out_off[-1]), dtype=torch.complex64, device=dev)
    xb = torch.empty_like(x)
    assert lib.adfft_execute_adjoint(h, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(xb.data_ptr()), ctypes.c_void_p(s)) == 0
    torch.cuda.synchronize()
    for i, (N, a) in enumerate(zip(Ns, alphas)):
        M = int(round(a * N))
        p = adfft.Plan(N, batch=1, dtype=adfft.R32, M=M)
        xi = x[in_off[i]:in_off[i + 1]].contiguous()
        Xi = torch.empty(M, dtype=torch.complex64, device=dev)
        p.execute(xi.data_ptr(), Xi.data_ptr())
        gi = g[out_off[i]:out_off[i + 1]].contiguous()
        xbi = torch.empty(N, device=dev)
        p.execute_adjoint(gi.data_ptr(), xbi.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(X[out_off[i]:out_off[i + 1]], Xi), (i, N, a)
        assert torch.equal(xb[in_off[i]:in_off[i + 1]], xbi), (i, N, a)
    lib.adfft_plan_destroy(h)


def test_ragged_workload_against_oracle():
    """10000 real fp32 signals (N = 2^e, e in 8..16, alpha in {2,3,4,8,2.5}): one
    graph-replayed forward, sampled signals and bins against the FP64 oracle."""
    torch = _torch()
    import ctypes
    x_np, Ns, alphas, offs = signals.ragged_r32()
    lib, h, in_off, out_off = make_ragged(torch, Ns, alphas)
    assert np.array_equal(in_off, offs)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(x_np).to(dev)
    X = torch.empty(int(out_off[-1]), dtype=torch.complex64, device=dev)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.adfft_execute(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(X.data_ptr()), s) == 0
    assert lib.adfft_execute(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(X.data_ptr()), s) == 0
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    pick = np.concatenate([rng.choice(np.where(Ns == n)[0], 2) for n in np.unique(Ns)])
    for i in pick:
        N, M = int(Ns[i]), int(round(alphas[i] * Ns[i]))
        bins = np.unique(rng.integers(0, M, 256))
        got = X[int(out_off[i]) + torch.from_numpy(bins).to(dev)].cpu().numpy()
        ref = oracle.alpha_dft(x_np[in_off[i]:in_off[i + 1]].astype(np.float64), M, bins=bins)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 2e-6 * np.log2(M), (i, N, alphas[i], err)
    lib.adfft_plan_destroy(h)


def test_ragged_loss_gradient():
    """loss = sum |X - Y|^2 over a ragged batch: the adjoint gives 2 Re(S A^H (X - Y)),
    checked per signal against the FP64 oracle's adjoint on a sub-batch."""
    torch = _torch()
    import ctypes
    rng = np.random.default_rng(9)
    Ns = [256, 1024, 4096, 512, 2048, 8192]
    alphas = [2.0, 8.0, 2.5, 3.0, 4.0, 2.5]
    lib, h, in_off, out_off = make_ragged(torch, Ns, alphas)
    dev = torch.device("cuda:0")
    x_np = rng.standard_normal(int(in_off[-1])).astype(np.float32)
    Y_np = ((rng.standard_normal(int(out_off[-1])) + 1j * rng.standard_normal(int(out_off[-1]))) * 0.01).astype(np.complex64)
    x = torch.from_numpy(x_np).to(dev)
    X = torch.empty(int(out_off[-1]), dtype=torch.complex64, device=dev)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.adfft_execute(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(X.data_ptr()), s) == 0
    gX = 2 * (X - torch.from_numpy(Y_np).to(dev))
    gx = torch.empty_like(x)
    assert lib.adfft_execute_adjoint(h, ctypes.c_void_p(gX.data_ptr()), ctypes.c_void_p(gx.data_ptr()), s) == 0
    torch.cuda.synchronize()
    for i, (N, a) in enumerate(zip(Ns, alphas)):
        M = int(round(a * N))
        xi = x_np[in_off[i]:in_off[i + 1]].astype(np.float64)
        Xi = oracle.alpha_dft(xi, M)
        ref = oracle.alpha_dft_adjoint(2 * (Xi - Y_np[out_off[i]:out_off[i + 1]]), N, real_input=True)
        got = gx[in_off[i]:in_off[i + 1]].cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-6 * np.log2(M)
    lib.adfft_plan_destroy(h)


def _c5_plan(torch):
    x_np, Ns, alphas, _ = signals.ragged_r32(count=10000)
    plan = adfft.RaggedPlan(Ns, alphas, adfft.R32)
    return x_np, np.asarray(Ns), np.asarray(alphas), plan


def test_ragged_c5_adjoint_every_class_against_oracle():
    """The 10000-signal ragged workload: the adjoint of one signal of every shape class
    (including the 16384-point classes with clusters of up to 16 CTAs and N = 65536) against
    the oracle's explicit adjoint on sampled output samples."""
    torch = _torch()
    x_np, Ns, alphas, plan = _c5_plan(torch)
    Ms = np.rint(alphas * Ns).astype(np.int64)
    rng = np.random.default_rng(21)
    dev = torch.device("cuda:0")
    g = torch.randn(int(plan.out_off[-1]), dtype=torch.complex64, device=dev)
    xb = torch.empty(int(plan.in_off[-1]), dtype=torch.float32, device=dev)
    plan.execute_adjoint(g.data_ptr(), xb.data_ptr())
    plan.sync_status()
    first = {}
    for i, key in enumerate(zip(Ns.tolist(), Ms.tolist())):
        first.setdefault(key, i)
    assert len(first) >= 40
    for (N, M), i in sorted(first.items()):
        gi = g[plan.out_off[i]:plan.out_off[i + 1]].cpu().numpy().astype(np.complex128)
        samples = np.unique(np.concatenate([[0, 1, N - 1, N // 2], rng.integers(0, N, 12)]))
        ref = oracle.alpha_dft_adjoint(gi, N, real_input=True, samples=samples)
        got = xb[plan.in_off[i]:plan.in_off[i + 1]][torch.from_numpy(samples).to(dev)].cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 2e-6 * np.log2(M), (N, M, err)


def test_ragged_c5_fp32_gradient_directional_difference():
    """FP32 gradient of L = sum |X_m - Y_m|^2 over the whole 10000-signal ragged workload
    (Y complex Gaussian): the central difference (L(x + e d) - L(x - e d)) / (2 e) along
    random +-1 directions, which is exact for a quadratic L up to rounding, against
    <grad, d> with grad = Re(A^H 2 (X - Y)) from the ragged adjoint.  One direction over
    every sample, and one confined to the signals of the N = 65536 classes."""
    torch = _torch()
    x_np, Ns, alphas, plan = _c5_plan(torch)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(x_np).to(dev)
    nb = int(plan.out_off[-1])
    gen = torch.Generator(device=dev).manual_seed(5)
    Y = torch.randn(nb, dtype=torch.complex64, device=dev, generator=gen)
    X = torch.empty(nb, dtype=torch.complex64, device=dev)

    def loss(xv):
        plan.execute(xv.data_ptr(), X.data_ptr())
        plan.sync_status()
        return (X - Y).abs().double().pow(2).sum().item()

    loss(x)
    gout = 2 * (X - Y)
    grad = torch.empty_like(x)
    plan.execute_adjoint(gout.data_ptr(), grad.data_ptr())
    plan.sync_status()
    big = torch.zeros_like(x)
    for i in np.flatnonzero(Ns == 65536):
        big[plan.in_off[i]:plan.in_off[i + 1]] = 1.0
    for mask in (None, big):
        d = torch.randint(0, 2, x.shape, device=dev, generator=gen).float() * 2 - 1
        if mask is not None:
            d = d * mask
        eps = 0.5
        fd = (loss(x + eps * d) - loss(x - eps * d)) / (2 * eps)
        an = (grad.double() * d.double()).sum().item()
        assert abs(fd - an) <= 1e-4 * abs(an), (fd, an)


@pytest.mark.parametrize("code,seed,count", [(adfft.R32, 11, 60), (adfft.C64, 12, 40), (adfft.R32, 13, 300)])
def test_ragged_queue_form_matches_class_graph(code, seed, count):
    """The persistent queue form (whole / fft / unpack tiles) against the class-graph form at
    every bin and against the oracle on sampled bins of one signal per class; mixes include
    N = 65536 signals (split into fft and unpack tiles)."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    Ns = [int(2 ** e) for e in rng.integers(8, 17, size=count)] + [65536, 65536, 256]
    alphas = list(rng.choice([2.0, 3.0, 4.0, 8.0, 2.5], size=len(Ns) - 3)) + [8.0, 2.5, 2.0]
    plan = adfft.RaggedPlan(Ns, alphas, code)
    dev = torch.device("cuda:0")
    ni, no = int(plan.in_off[-1]), int(plan.out_off[-1])
    x = torch.randn(ni, device=dev) if code == adfft.R32 else torch.randn(ni, dtype=torch.complex64, device=dev)
    Xg = torch.empty(no, dtype=torch.complex64, device=dev)
    plan.set_form(adfft.RAGGED_CLASSES)
    plan.execute(x.data_ptr(), Xg.data_ptr())
    plan.sync_status()
    plan.set_form(adfft.RAGGED_QUEUE)
    Xq = torch.full((no,), complex(float("nan"), float("nan")), dtype=torch.complex64, device=dev)
    for _ in range(2):   # the second execute replays the captured graph (counters reset inside)
        plan.execute(x.data_ptr(), Xq.data_ptr())
        plan.sync_status()
    assert torch.isfinite(Xq.view(torch.float32)).all().item()
    assert (torch.linalg.vector_norm(Xq - Xg) / torch.linalg.vector_norm(Xg)).item() <= 1e-6
    xs = x.cpu().numpy()
    seen = set()
    for i, (N, a) in enumerate(zip(Ns, alphas)):
        M = int(round(a * N))
        if (N, M) in seen:
            continue
        seen.add((N, M))
        bins = np.unique(np.concatenate([[0, M // 2, M - 1], rng.integers(0, M, 64)]))
        xi = xs[plan.in_off[i]:plan.in_off[i + 1]]
        ref = oracle.alpha_dft(xi.astype(np.complex128 if code == adfft.C64 else np.float64), M, bins=bins)
        got = Xq[int(plan.out_off[i]):int(plan.out_off[i + 1])][torch.from_numpy(bins).to(dev)].cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-6 * np.log2(M), (N, M)


def test_ragged_queue_form_c5_every_class():
    """The 10000-signal workload through the queue form: every bin against the class graph,
    and one signal per shape class against the oracle on sampled bins."""
    torch = _torch()
    x_np, Ns, alphas, plan = _c5_plan(torch)
    Ms = np.rint(alphas * Ns).astype(np.int64)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(x_np).to(dev)
    no = int(plan.out_off[-1])
    Xg = torch.empty(no, dtype=torch.complex64, device=dev)
    plan.set_form(adfft.RAGGED_CLASSES)
    plan.execute(x.data_ptr(), Xg.data_ptr())
    plan.set_form(adfft.RAGGED_QUEUE)
    Xq = torch.empty(no, dtype=torch.complex64, device=dev)
    plan.execute(x.data_ptr(), Xq.data_ptr())
    plan.sync_status()
    assert (torch.linalg.vector_norm(Xq - Xg) / torch.linalg.vector_norm(Xg)).item() <= 1e-6
    rng = np.random.default_rng(8)
    first = {}
    for i, key in enumerate(zip(Ns.tolist(), Ms.tolist())):
        first.setdefault(key, i)
    for (N, M), i in sorted(first.items()):
        bins = np.unique(np.concatenate([[0, M // 2, M - 1], rng.integers(0, M, 48)]))
        ref = oracle.alpha_dft(x_np[plan.in_off[i]:plan.in_off[i + 1]].astype(np.float64), M, bins=bins)
        got = Xq[int(plan.out_off[i]):int(plan.out_off[i + 1])][torch.from_numpy(bins).to(dev)].cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-6 * np.log2(M), (N, M)


def test_ragged_queue_form_refused_where_unavailable():
    _torch()
    plan = adfft.RaggedPlan([1000, 2000], [2.5, 2.5], adfft.C64)   # chirp-z classes: no fold geometry
    with pytest.raises(adfft.AdfftError):
        plan.set_form(adfft.RAGGED_QUEUE)
    with pytest.raises(adfft.AdfftError):
        adfft.RaggedPlan([3, 4], [2.0, 2.0], adfft.R32)             # even-N signal at an odd offset
