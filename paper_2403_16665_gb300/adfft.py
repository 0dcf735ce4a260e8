"""Thin ctypes binding of the adfft C ABI (include/adfft.h).

Argument marshalling only: every step of the transform runs in the CUDA
kernels of libadfft.so.  torch supplies device memory and streams.  There is
no CPU fallback: if the library is missing or no GPU is present, calls fail
loudly.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libadfft.so")

# adfft_dtype_t
R32, C64, R64, C128 = 0, 1, 2, 3
# adfft_algo_t
ALGO_AUTO, ALGO_FOLD, ALGO_BLUESTEIN, ALGO_FOUR_STEP = 0, 1, 2, 3
# adfft_precision_t
PREC_NATIVE, PREC_FP16X2, PREC_BF16X3 = 0, 1, 2
# adfft_plan_autotune flags
TUNE_WITH_ADJOINT = 1
# adfft_output_t
OUTPUT_FULL, OUTPUT_HALF = 0, 1
# adfft_ragged_form_t
RAGGED_CLASSES, RAGGED_QUEUE = 0, 1

STATUS = {
    0: "ADFFT_OK", -1: "ADFFT_ERR_INVALID_ARG", -2: "ADFFT_ERR_INVALID_ALPHA",
    -3: "ADFFT_ERR_UNSUPPORTED_SIZE", -4: "ADFFT_ERR_MISALIGNED", -5: "ADFFT_ERR_OVERLAP",
    -6: "ADFFT_ERR_CUDA", -7: "ADFFT_ERR_OOM", -8: "ADFFT_ERR_TIMEOUT",
    -9: "ADFFT_ERR_NOT_SUPPORTED",
}

# every symbol include/adfft.h declares (the ABI test checks the library exports them)
EXPORTS = (
    "adfft_plan_create", "adfft_plan_create_bins", "adfft_plan_create_ragged",
    "adfft_plan_offsets", "adfft_last_error", "adfft_status_string", "adfft_plan_destroy",
    "adfft_plan_set_scale", "adfft_plan_set_algorithm", "adfft_plan_set_precision",
    "adfft_plan_get_info", "adfft_plan_workspace_bytes", "adfft_execute",
    "adfft_execute_adjoint", "adfft_execute_host", "adfft_plan_sync_status",
    "adfft_execute_noalloc", "adfft_plan_autotune", "adfft_autotune_save", "adfft_autotune_load",
    "adfft_autotune_clear", "adfft_plan_set_launch_shape", "adfft_plan_set_output",
    "adfft_plan_set_ragged_form", "adfft_ragged_queue_layout",
)


class AdfftError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s%s" % (what + ": " if what else "", STATUS.get(code, str(code))))


class PlanInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("M", ctypes.c_int64), ("batch", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("algo", ctypes.c_int32), ("fft_len", ctypes.c_int64),
                ("residues", ctypes.c_int64), ("fold", ctypes.c_int64), ("cluster", ctypes.c_int32),
                ("passes", ctypes.c_int32), ("scale", ctypes.c_double), ("staged", ctypes.c_int32),
                ("tuned", ctypes.c_int32), ("grid", ctypes.c_int32), ("four_step_a", ctypes.c_int32),
                ("out_bins", ctypes.c_int64)]


_lib = None


def load(path: str | None = None):
    """Load libadfft.so (build it first with paper_2403_16665_gb300._build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libadfft.so is not built (%s); run __graft_entry__.build()" % p)
    lib = ctypes.CDLL(p)
    i64, i32, f64, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "adfft_plan_create": ([i64, f64, i64, i32], vp),
        "adfft_plan_create_bins": ([i64, i64, i64, i32], vp),
        "adfft_plan_create_ragged": ([vp, vp, i64, i32], vp),
        "adfft_plan_offsets": ([vp, vp, vp], i32),
        "adfft_last_error": ([], i32),
        "adfft_status_string": ([i32], ctypes.c_char_p),
        "adfft_plan_destroy": ([vp], i32),
        "adfft_plan_set_scale": ([vp, f64], i32),
        "adfft_plan_set_algorithm": ([vp, i32], i32),
        "adfft_plan_set_precision": ([vp, i32], i32),
        "adfft_plan_set_output": ([vp, i32], i32),
        "adfft_plan_set_ragged_form": ([vp, i32], i32),
        "adfft_plan_get_info": ([vp, ctypes.POINTER(PlanInfo)], i32),
        "adfft_plan_workspace_bytes": ([vp], ctypes.c_size_t),
        "adfft_execute": ([vp, vp, vp, vp], i32),
        "adfft_execute_adjoint": ([vp, vp, vp, vp], i32),
        "adfft_execute_host": ([vp, vp, vp, vp], i32),
        "adfft_plan_sync_status": ([vp, vp], i32),
        "adfft_execute_noalloc": ([i64, i64, i64, i32, vp, vp, vp], i32),
        "adfft_plan_autotune": ([vp, vp, vp, vp, i32, i32], i32),
        "adfft_autotune_save": ([ctypes.c_char_p], i32),
        "adfft_autotune_load": ([ctypes.c_char_p], i32),
        "adfft_autotune_clear": ([], i32),
        "adfft_plan_set_launch_shape": ([vp, i64, i32, i32, i32], i32),
        "adfft_ragged_queue_layout": ([vp, vp, i64, i32, i32, vp, i64, vp, vp, i64, vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc, what):
    if rc != 0:
        raise AdfftError(rc, what)


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """Owning wrapper of an adfft_plan_t (the C calls, one to one)."""

    def __init__(self, N, alpha=None, batch=1, dtype=R32, M=None):
        lib = load()
        if M is not None:
            h = lib.adfft_plan_create_bins(int(N), int(M), int(batch), int(dtype))
        else:
            h = lib.adfft_plan_create(int(N), float(alpha), int(batch), int(dtype))
        if not h:
            raise AdfftError(lib.adfft_last_error(), "adfft_plan_create")
        self._h = ctypes.c_void_p(h)
        self.lib = lib
        self.info = self.get_info()

    @property
    def handle(self):
        return self._h

    def get_info(self) -> PlanInfo:
        info = PlanInfo()
        _check(self.lib.adfft_plan_get_info(self._h, ctypes.byref(info)), "adfft_plan_get_info")
        return info

    def set_scale(self, S):
        _check(self.lib.adfft_plan_set_scale(self._h, float(S)), "adfft_plan_set_scale")
        self.info = self.get_info()

    def set_algorithm(self, algo):
        _check(self.lib.adfft_plan_set_algorithm(self._h, int(algo)), "adfft_plan_set_algorithm")
        self.info = self.get_info()

    def set_precision(self, mode):
        _check(self.lib.adfft_plan_set_precision(self._h, int(mode)), "adfft_plan_set_precision")
        self.info = self.get_info()

    def set_output(self, mode):
        """OUTPUT_FULL (all M bins) or OUTPUT_HALF (real input: bins 0 .. M/2)."""
        _check(self.lib.adfft_plan_set_output(self._h, int(mode)), "adfft_plan_set_output")
        self.info = self.get_info()

    def set_launch_shape(self, fft_len=0, cluster=0, staged=-1, grid=0):
        _check(self.lib.adfft_plan_set_launch_shape(self._h, int(fft_len), int(cluster), int(staged), int(grid)),
               "adfft_plan_set_launch_shape")
        self.info = self.get_info()

    def workspace_bytes(self) -> int:
        return int(self.lib.adfft_plan_workspace_bytes(self._h))

    def execute(self, d_in: int, d_out: int, stream=None):
        _check(self.lib.adfft_execute(self._h, ctypes.c_void_p(d_in), ctypes.c_void_p(d_out),
                                      ctypes.c_void_p(_stream_handle(stream))), "adfft_execute")

    def execute_adjoint(self, d_grad_out: int, d_grad_in: int, stream=None):
        _check(self.lib.adfft_execute_adjoint(self._h, ctypes.c_void_p(d_grad_out),
                                              ctypes.c_void_p(d_grad_in),
                                              ctypes.c_void_p(_stream_handle(stream))),
               "adfft_execute_adjoint")

    def execute_host(self, h_in: int, h_out: int, stream=None):
        _check(self.lib.adfft_execute_host(self._h, ctypes.c_void_p(h_in), ctypes.c_void_p(h_out),
                                           ctypes.c_void_p(_stream_handle(stream))),
               "adfft_execute_host")

    def autotune(self, d_in: int, d_out: int, stream=None, iters=0, with_adjoint=False):
        """Time the candidate launch shapes on these buffers and keep the fastest (d_out is
        overwritten); with_adjoint: time forward + adjoint steps (training)."""
        _check(self.lib.adfft_plan_autotune(self._h, ctypes.c_void_p(d_in), ctypes.c_void_p(d_out),
                                            ctypes.c_void_p(_stream_handle(stream)), int(iters),
                                            TUNE_WITH_ADJOINT if with_adjoint else 0),
               "adfft_plan_autotune")
        self.info = self.get_info()

    def sync_status(self, stream=None):
        """Synchronise the stream and raise if a kernel of the plan reported an error."""
        _check(self.lib.adfft_plan_sync_status(self._h, ctypes.c_void_p(_stream_handle(stream))),
               "adfft_plan_sync_status")

    def destroy(self):
        if self._h is not None and self._h.value:
            self.lib.adfft_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class RaggedPlan(Plan):
    """adfft_plan_create_ragged: signals of uneven N and alpha packed back to back.

    in_off / out_off (numpy int64, count + 1 entries) are the packed offsets in
    samples and bins from adfft_plan_offsets.
    """

    def __init__(self, Ns, alphas, dtype=R32):
        import numpy as np
        lib = load()
        Na = np.ascontiguousarray(np.asarray(Ns, dtype=np.int64))
        Aa = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
        if Na.shape != Aa.shape or Na.ndim != 1:
            raise ValueError("Ns and alphas must be 1-D arrays of equal length")
        h = lib.adfft_plan_create_ragged(Na.ctypes.data_as(ctypes.c_void_p), Aa.ctypes.data_as(ctypes.c_void_p),
                                         int(Na.size), int(dtype))
        if not h:
            raise AdfftError(lib.adfft_last_error(), "adfft_plan_create_ragged")
        self._h = ctypes.c_void_p(h)
        self.lib = lib
        self.info = self.get_info()
        self.in_off = np.zeros(Na.size + 1, dtype=np.int64)
        self.form = None
        self.out_off = np.zeros(Na.size + 1, dtype=np.int64)
        _check(lib.adfft_plan_offsets(self._h, self.in_off.ctypes.data_as(ctypes.c_void_p),
                                      self.out_off.ctypes.data_as(ctypes.c_void_p)), "adfft_plan_offsets")


def _ragged_set_form(self, form):
    """RAGGED_CLASSES (graph of per-class launches) or RAGGED_QUEUE (one persistent kernel)."""
    _check(self.lib.adfft_plan_set_ragged_form(self._h, int(form)), "adfft_plan_set_ragged_form")
    self.form = int(form)


RaggedPlan.set_form = _ragged_set_form


def ragged_queue_layout(Ns, alphas, dtype=R32, lag=608):
    """adfft_ragged_queue_layout: the queue form's tiles for these shapes, computed on the host
    (no device needed).  Returns (tiles, whole): tiles an (n, 5) int32 array of (kind, class,
    signal or first whole index, a0, a1), whole the signals of the whole tiles in order."""
    import numpy as np
    lib = load()
    N = np.ascontiguousarray(np.asarray(Ns, dtype=np.int64))
    A = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    nt, nw = ctypes.c_int64(0), ctypes.c_int64(0)
    args = (N.ctypes.data_as(ctypes.c_void_p), A.ctypes.data_as(ctypes.c_void_p), int(N.size), int(dtype), int(lag))
    _check(lib.adfft_ragged_queue_layout(*args, None, 0, ctypes.byref(nt), None, 0, ctypes.byref(nw)),
           "adfft_ragged_queue_layout")
    tiles = np.zeros((max(nt.value, 1), 5), dtype=np.int32)
    whole = np.zeros(max(nw.value, 1), dtype=np.int64)
    _check(lib.adfft_ragged_queue_layout(*args, tiles.ctypes.data_as(ctypes.c_void_p), nt.value, ctypes.byref(nt),
                                         whole.ctypes.data_as(ctypes.c_void_p), nw.value, ctypes.byref(nw)),
           "adfft_ragged_queue_layout")
    return tiles[:nt.value], whole[:nw.value]


def autotune_save(path):
    """Write the process-wide tuning cache to a JSON file."""
    _check(load().adfft_autotune_save(os.fsencode(path)), "adfft_autotune_save")


def autotune_load(path):
    """Merge a tuning-cache file written by autotune_save."""
    _check(load().adfft_autotune_load(os.fsencode(path)), "adfft_autotune_load")


def autotune_clear():
    _check(load().adfft_autotune_clear(), "adfft_autotune_clear")


def execute_noalloc(N, M, batch, dtype, d_in: int, d_out: int, stream=None):
    """adfft_execute_noalloc: forward transform with no device allocation (R32 / C64)."""
    _check(load().adfft_execute_noalloc(int(N), int(M), int(batch), int(dtype), ctypes.c_void_p(d_in),
                                        ctypes.c_void_p(d_out), ctypes.c_void_p(_stream_handle(stream))),
           "adfft_execute_noalloc")


def _dtype_code(t):
    import torch
    return {torch.float32: R32, torch.complex64: C64, torch.float64: R64,
            torch.complex128: C128}[t]


def out_dtype(t):
    import torch
    return torch.complex128 if t in (torch.float64, torch.complex128) else torch.complex64


def alpha_dft(x, alpha=None, M=None, scale=None, algorithm=ALGO_AUTO, plan_cache=None):
    """X[b, m] = S sum_n x[b, n] exp(-2 pi i m n / M) for a CUDA tensor x [batch, N] or [N].

    alpha (or M = alpha*N) sets the bin count; scale S defaults to 1/N (T/N, T = 1).
    """
    import torch
    if not x.is_cuda:
        raise RuntimeError("alpha_dft needs a CUDA tensor (no CPU path)")
    one = x.dim() == 1
    x2 = x.reshape(1, -1) if one else x
    x2 = x2.contiguous()
    B, N = x2.shape
    if M is None:
        M = int(round(float(alpha) * N))
    key = (N, M, B, x2.dtype, scale, algorithm, x2.device.index)
    plan = plan_cache.get(key) if plan_cache is not None else None
    if plan is None:
        with torch.cuda.device(x2.device):
            plan = Plan(N, batch=B, dtype=_dtype_code(x2.dtype), M=M)
            if scale is not None:
                plan.set_scale(scale)
            if algorithm != ALGO_AUTO:
                plan.set_algorithm(algorithm)
        if plan_cache is not None:
            plan_cache[key] = plan
    X = torch.empty((B, M), dtype=out_dtype(x2.dtype), device=x2.device)
    plan.execute(x2.data_ptr(), X.data_ptr(), torch.cuda.current_stream(x2.device))
    return X[0] if one else X
