"""CPU checks of the C ABI: the library builds, loads, exports every symbol the
header declares, and rejects invalid arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

from paper_2403_16665_gb300 import _build, adfft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "adfft.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return adfft.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(adfft_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(adfft.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code, name in adfft.STATUS.items():
        assert lib.adfft_status_string(code).decode() == name
    assert lib.adfft_status_string(12345).decode() == "ADFFT_ERR_UNKNOWN"


@pytest.mark.parametrize("N,alpha,batch,dtype,code", [
    (0, 2.0, 1, 0, -1),            # N < 1
    (-5, 2.0, 1, 0, -1),
    (16, 2.0, -1, 0, -1),          # batch < 0
    (16, 2.0, 1, 7, -1),           # bad dtype
    (16, float("nan"), 1, 0, -2),  # alpha not finite
    (16, float("inf"), 1, 0, -2),
    (16, -1.0, 1, 0, -2),          # alpha <= 0
    (16, 0.0, 1, 0, -2),
    (10, 0.33, 1, 0, -2),          # alpha*N not an integer
    (8192, 2.5001, 1, 1, -2),
])
def test_create_rejects_invalid_arguments(lib, N, alpha, batch, dtype, code):
    h = lib.adfft_plan_create(N, alpha, batch, dtype)
    assert not h
    assert lib.adfft_last_error() == code


def test_null_plan_calls(lib):
    assert lib.adfft_plan_destroy(None) == 0
    assert lib.adfft_execute(None, None, None, None) == -1
    assert lib.adfft_execute_adjoint(None, None, None, None) == -1
    assert lib.adfft_execute_host(None, None, None, None) == -1
    assert lib.adfft_plan_set_scale(None, 1.0) == -1
    assert lib.adfft_plan_get_info(None, None) == -1
    assert lib.adfft_plan_offsets(None, None, None) == -1
    assert lib.adfft_plan_workspace_bytes(None) == 0


def test_create_without_gpu_reports_cuda_error(lib):
    """On a machine with no GPU a valid request fails cleanly with ADFFT_ERR_CUDA."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = lib.adfft_plan_create(1024, 4.0, 1, 2)
    assert not h
    assert lib.adfft_last_error() == -6


def test_bindings_refuse_cpu_tensors():
    import torch
    with pytest.raises(RuntimeError):
        adfft.alpha_dft(torch.zeros(16), alpha=2)


def test_fastdiv_magic_matches_integer_division():
    """Host-side magic numbers of the kernels' division by an invariant (fft_device.cuh)."""
    def magic(d):
        l = 0
        while (1 << l) < d:
            l += 1
        return ((1 << 32) * ((1 << l) - d)) // d + 1, l

    import random
    rnd = random.Random(7)
    for d in [1, 2, 3, 5, 7, 15, 16, 17, 100, 255, 4096, 30720, 65535]:
        mul, sh = magic(d)
        assert mul < (1 << 32)
        for n in [0, 1, d - 1, d, d + 1, 2**31 - 1] + [rnd.randrange(0, 2**31) for _ in range(200)]:
            q = (((n * mul) >> 32) + n) >> sh
            assert q == n // d, (d, n)
