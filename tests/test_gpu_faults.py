"""Failure paths without a GPU fault: host-side injection through ADFFT_FAULT (read when a
plan is created).

- alloc:<k>: the k-th device allocation of plan creation fails; creation reports out of
  memory, frees what it had allocated, and a later creation succeeds.
- launch: every launch of the plan fails; the call reports ADFFT_ERR_CUDA and nothing is
  written.
- copy_skip:<s>: the fused kernel never issues the input copy of signal s; its bounded wait
  (shortened to ~10 ms for the test) runs out, the kernel returns, the plan reports
  ADFFT_ERR_TIMEOUT, the cluster that owned signal s transforms no later signal, every other
  signal is exact, and the context stays usable.
"""
import numpy as np
import pytest

from paper_2403_16665_gb300 import adfft, signals

pytestmark = pytest.mark.gpu

N, ALPHA = 16384, 8
M = N * ALPHA


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    adfft.load()
    return torch


@pytest.fixture
def fault_env(monkeypatch):
    def set_fault(v):
        monkeypatch.setenv("ADFFT_FAULT", v)
    yield set_fault
    monkeypatch.delenv("ADFFT_FAULT", raising=False)


# (N, M, batch, k): the single-pass plan allocates its status word and twiddle table; the
# two-pass plan (N = 2^22, alpha = 16) also its pass tables and a 256 MiB workspace (the 6th)
@pytest.mark.parametrize("n,m,batch,k", [(N, M, 64, 1), (N, M, 64, 2), (1 << 22, 1 << 26, 1, 3),
                                         (1 << 22, 1 << 26, 1, 6)])
def test_allocation_fault_reports_oom_and_frees(fault_env, n, m, batch, k):
    torch = _torch()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    fault_env("alloc:%d" % k)
    with pytest.raises(adfft.AdfftError) as ei:
        adfft.Plan(n, batch=batch, dtype=adfft.R32, M=m)
    assert ei.value.code == -7              # ADFFT_ERR_OOM
    assert adfft.load().adfft_last_error() == -7
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) <= (8 << 20)  # nothing of the failed creation stays allocated
    fault_env("")
    p = adfft.Plan(n, batch=batch, dtype=adfft.R32, M=m)
    assert p.info.M == m


def test_launch_fault_launches_nothing(fault_env):
    torch = _torch()
    fault_env("launch")
    plan = adfft.Plan(N, batch=4, dtype=adfft.R32, M=M)
    x = torch.randn((4, N), device="cuda")
    X = torch.full((4, M), complex(float("nan"), float("nan")), dtype=torch.complex64, device="cuda")
    with pytest.raises(adfft.AdfftError) as ei:
        plan.execute(x.data_ptr(), X.data_ptr())
    assert ei.value.code == -6              # ADFFT_ERR_CUDA
    xb = torch.full_like(x, float("nan"))
    with pytest.raises(adfft.AdfftError):
        plan.execute_adjoint(X.data_ptr(), xb.data_ptr())
    torch.cuda.synchronize()
    assert torch.isnan(X.view(torch.float32)).all().item() and torch.isnan(xb).all().item()


def test_skipped_copy_times_out_and_kernel_returns(fault_env):
    torch = _torch()
    B, skip = 64, 5
    x_np, _ = signals.batch_r32(batch=B, N=N, alpha=ALPHA, seed=9)
    x = torch.from_numpy(x_np).cuda()
    clean = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    clean.set_launch_shape(N // 2, 4, 1, 0)
    Xc = torch.empty((B, M), dtype=torch.complex64, device="cuda")
    clean.execute(x.data_ptr(), Xc.data_ptr())
    clean.sync_status()

    fault_env("copy_skip:%d" % skip)
    plan = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    plan.set_launch_shape(N // 2, 4, 1, 0)       # staged input: each signal arrives by a bulk copy
    info = plan.info
    assert info.staged == 1
    X = torch.full((B, M), complex(float("nan"), float("nan")), dtype=torch.complex64, device="cuda")
    plan.execute(x.data_ptr(), X.data_ptr())
    with pytest.raises(adfft.AdfftError) as ei:
        plan.sync_status()
    assert ei.value.code == -8                   # ADFFT_ERR_TIMEOUT
    # the cluster that owned signal `skip` stops: that signal and its later ones stay unwritten
    grid = info.grid
    owned = [s for s in range(B) if s % grid == skip % grid]
    later = [s for s in owned if s >= skip]
    for s in later:
        assert torch.isnan(X[s].view(torch.float32)).all().item(), s
    others = [s for s in range(B) if s not in later]
    idx = torch.tensor(others, device="cuda")
    assert torch.equal(X[idx], Xc[idx])
    # the status word was cleared by the read, and the context still works
    fault_env("")
    again = adfft.Plan(N, batch=B, dtype=adfft.R32, M=M)
    again.set_launch_shape(N // 2, 4, 1, 0)
    X2 = torch.empty_like(X)
    again.execute(x.data_ptr(), X2.data_ptr())
    again.sync_status()
    assert torch.equal(X2, Xc)
