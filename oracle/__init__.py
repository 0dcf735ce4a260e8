"""FP64 CPU oracle for the alpha-densified DFT (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package.  The product path
(``paper_2403_16665_gb300``) never imports it and shares no code with it.

``alpha_dft`` evaluates Eq. 7 of the paper by direct summation,
    X_m = S * sum_n x_n exp(-2 pi i m n / M),  m = 0..M-1,  M = alpha*N,
with the scale S = T/N of Eq. 2 (S = 1 gives Eq. 7 as printed); see
``adfft_oracle.c`` for the arithmetic.  ``alpha_dft_adjoint`` is the conjugate
transpose of the same matrix times S.  Parity of this oracle is pinned by the
``-m "not gpu"`` tests against closed forms, numpy's FFT of the zero-padded
signal (Sec. 2: alpha > 1 equals appending (alpha-1)N zeros) and brute force
in extended precision.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adfft_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc + OpenMP into oracle/_lib/liboracle.so."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, f64 = ctypes.c_int64, ctypes.c_double
            p = ctypes.c_void_p
            lib.oracle_alpha_dft.argtypes = [i64, i64, i64, f64, p, p, p, i64, p, p, ctypes.c_int]
            lib.oracle_alpha_dft.restype = ctypes.c_int
            lib.oracle_alpha_dft_adjoint.argtypes = [i64, i64, i64, f64, p, p, p, p, ctypes.c_int]
            lib.oracle_alpha_dft_adjoint.restype = ctypes.c_int
            lib.oracle_alpha_dft_adjoint_samples.argtypes = [i64, i64, i64, f64, p, p, p, i64, p, p, ctypes.c_int]
            lib.oracle_alpha_dft_adjoint_samples.restype = ctypes.c_int
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    """Threads the oracle's OpenMP runtime uses by default."""
    return int(_load().oracle_max_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def output_bins(N: int, alpha) -> int:
    """M = alpha*N; alpha*N must be an integer (Eq. 6: m = 0..alpha N - 1)."""
    M = float(alpha) * N
    Mi = int(round(M))
    if abs(M - Mi) > 1e-9 * max(1.0, M) or Mi < 1:
        raise ValueError("alpha*N must be a positive integer")
    return Mi


def alpha_dft(x, M: int, S: float | None = None, bins=None, threads: int = 0):
    """Direct-sum Eq. 7 for a batch.

    x: real or complex array [N] or [batch, N]; M: number of output bins;
    S: scale (default T/N with T = 1); bins: optional int array of bin indices.
    Returns complex128 [batch, nbins] (or [nbins] for 1-D x).
    """
    x = np.asarray(x)
    one = x.ndim == 1
    x2 = x.reshape(1, -1) if one else x
    B, N = x2.shape
    S = (1.0 / N) if S is None else float(S)
    xr = np.ascontiguousarray(x2.real, dtype=np.float64)
    xi = np.ascontiguousarray(x2.imag, dtype=np.float64) if np.iscomplexobj(x2) else None
    if bins is None:
        b_arr, nb = None, int(M)
    else:
        b_arr = np.ascontiguousarray(np.asarray(bins, dtype=np.int64))
        if b_arr.size and (b_arr.min() < 0 or b_arr.max() >= M):
            raise ValueError("bin index out of range")
        nb = int(b_arr.size)
    Xr = np.empty((B, nb), dtype=np.float64)
    Xi = np.empty((B, nb), dtype=np.float64)
    rc = _load().oracle_alpha_dft(B, N, int(M), S, _ptr(xr), _ptr(xi), _ptr(b_arr), nb,
                                  _ptr(Xr), _ptr(Xi), int(threads))
    if rc != 0:
        raise ValueError("oracle_alpha_dft rejected its arguments")
    X = Xr + 1j * Xi
    return X[0] if one else X


def alpha_dft_adjoint(g, N: int, S: float | None = None, real_input: bool = False,
                      threads: int = 0, samples=None):
    """Conjugate transpose of Eq. 7 times S: xb_n = S sum_m exp(+2 pi i m n/M) g_m.

    g: complex array [M] or [batch, M].  For a real-input forward map the
    adjoint with respect to the real inner product is the real part, which is
    returned when real_input is True.  samples: optional int array of output
    indices n (0 <= n < N); the result then holds those samples only, in that
    order ([nsamples] or [batch, nsamples]).
    """
    g = np.asarray(g)
    one = g.ndim == 1
    g2 = g.reshape(1, -1) if one else g
    B, M = g2.shape
    S = (1.0 / N) if S is None else float(S)
    gr = np.ascontiguousarray(g2.real, dtype=np.float64)
    gi = np.ascontiguousarray(g2.imag, dtype=np.float64)
    if samples is not None:
        smp = np.ascontiguousarray(np.asarray(samples, dtype=np.int64))
        if smp.size and (smp.min() < 0 or smp.max() >= N):
            raise ValueError("sample index out of range")
        xr = np.empty((B, smp.size), dtype=np.float64)
        xi = np.empty((B, smp.size), dtype=np.float64)
        rc = _load().oracle_alpha_dft_adjoint_samples(B, int(N), M, S, _ptr(gr), _ptr(gi), _ptr(smp),
                                                      int(smp.size), _ptr(xr), _ptr(xi), int(threads))
    else:
        xr = np.empty((B, N), dtype=np.float64)
        xi = np.empty((B, N), dtype=np.float64)
        rc = _load().oracle_alpha_dft_adjoint(B, int(N), M, S, _ptr(gr), _ptr(gi), _ptr(xr),
                                              _ptr(xi), int(threads))
    if rc != 0:
        raise ValueError("oracle_alpha_dft_adjoint rejected its arguments")
    out = xr if real_input else xr + 1j * xi
    return out[0] if one else out
