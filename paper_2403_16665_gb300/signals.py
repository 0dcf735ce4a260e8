"""Seeded synthetic input signals (no transform arithmetic lives here).

Shared by the tests, the benchmark and the oracle checks: it only draws the
test signals of the paper's kind (sampled tones plus Gaussian noise, sampled
at t_n = nT/N as in Eq. 3 with T = 1).  Frequencies are drawn "off the bins":
a tone of nu cycles per record is rejected when alpha*nu lies within 0.05 of
an integer, so it falls neither on the 1/T grid nor on the finer 1/(alpha T)
grid of Eq. 6.

Workloads (name -> recipe):
  single_r64   1 real fp64 signal, N=1024, alpha=4: 3 cosines A~U(0.5,2),
               nu~U(0,N/2), phase~U(0,2pi), noise sigma=0.1.  Seed 1.
  batch_r32    4096 real fp32 signals, N=16384, alpha=8: 5 cosines
               A~U(0.1,1), nu~U(0,N/2), noise sigma=0.2.  Seed 2.
  batch_c64    1024 complex64 signals, N=8192, alpha in {2.5, 3.75}: 5 complex
               exponentials A~U(0.1,1), nu~U(0,N), complex noise E|w|^2=0.1^2.
               Seed 3.
  large_r32    8 real fp32 signals, N=2^22, alpha=16: 20 cosines with A
               log-uniform on [1e-4, 1], noise sigma=1e-3.  Seed 4.
  ragged_r32   10000 real fp32 signals, N=2^e with e~U{8..16},
               alpha~U{2,3,4,8,2.5}, signals as in batch_r32.  Seed 5.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _off_grid(rng, count, lo, hi, alpha, min_gap=0.05):
    """Draw `count` frequencies nu ~ U(lo, hi) with alpha*nu >= min_gap from any integer."""
    out = np.empty(count)
    k = 0
    while k < count:
        v = rng.uniform(lo, hi, size=2 * (count - k) + 4)
        a = alpha * v
        v = v[np.abs(a - np.round(a)) >= min_gap]
        take = min(count - k, v.size)
        out[k:k + take] = v[:take]
        k += take
    return out


def real_tones(batch, N, alpha, n_tones, amp, noise_sigma, seed, dtype=np.float32,
               log_amp=False, chunk=256):
    """[batch, N] real signals: sum of cosines A cos(2 pi nu n/N + phi) + N(0, sigma^2).

    amp = (lo, hi); with log_amp the amplitudes are log-uniform on [lo, hi].
    Returns (x, params) with params = dict(nu, A, phi) arrays [batch, n_tones].
    """
    rng = _rng(seed)
    nu = _off_grid(rng, batch * n_tones, 0.0, N / 2, alpha).reshape(batch, n_tones)
    if log_amp:
        A = np.exp(rng.uniform(np.log(amp[0]), np.log(amp[1]), size=(batch, n_tones)))
    else:
        A = rng.uniform(amp[0], amp[1], size=(batch, n_tones))
    phi = rng.uniform(0.0, 2 * np.pi, size=(batch, n_tones))
    x = np.empty((batch, N), dtype=dtype)
    n = np.arange(N, dtype=np.float64)
    for b0 in range(0, batch, chunk):
        b1 = min(batch, b0 + chunk)
        acc = np.zeros((b1 - b0, N), dtype=np.float64)
        for t in range(n_tones):
            ph = (2 * np.pi / N) * nu[b0:b1, t, None] * n[None, :] + phi[b0:b1, t, None]
            acc += A[b0:b1, t, None] * np.cos(ph)
        acc += noise_sigma * rng.standard_normal(size=(b1 - b0, N))
        x[b0:b1] = acc
    return x, dict(nu=nu, A=A, phi=phi)


def complex_tones(batch, N, alpha, n_tones, amp, noise_sigma, seed, dtype=np.complex64,
                  chunk=256):
    """[batch, N] complex signals: sum of A exp(i(2 pi nu n/N + phi)) + complex noise.

    nu ~ U(0, N) off the alpha-grid; the complex noise has E|w|^2 = sigma^2
    (each of the real and imaginary parts has standard deviation sigma/sqrt 2).
    """
    rng = _rng(seed)
    nu = _off_grid(rng, batch * n_tones, 0.0, float(N), alpha).reshape(batch, n_tones)
    A = rng.uniform(amp[0], amp[1], size=(batch, n_tones))
    phi = rng.uniform(0.0, 2 * np.pi, size=(batch, n_tones))
    x = np.empty((batch, N), dtype=dtype)
    n = np.arange(N, dtype=np.float64)
    s = noise_sigma / np.sqrt(2.0)
    for b0 in range(0, batch, chunk):
        b1 = min(batch, b0 + chunk)
        acc = np.zeros((b1 - b0, N), dtype=np.complex128)
        for t in range(n_tones):
            ph = (2 * np.pi / N) * nu[b0:b1, t, None] * n[None, :] + phi[b0:b1, t, None]
            acc += A[b0:b1, t, None] * np.exp(1j * ph)
        acc += s * (rng.standard_normal(size=(b1 - b0, N))
                    + 1j * rng.standard_normal(size=(b1 - b0, N)))
        x[b0:b1] = acc
    return x, dict(nu=nu, A=A, phi=phi)


def single_r64(batch=1, N=1024, alpha=4, seed=1):
    return real_tones(batch, N, alpha, 3, (0.5, 2.0), 0.1, seed, dtype=np.float64)


def batch_r32(batch=4096, N=16384, alpha=8, seed=2):
    return real_tones(batch, N, alpha, 5, (0.1, 1.0), 0.2, seed, dtype=np.float32)


def batch_c64(batch=1024, N=8192, alpha=2.5, seed=3):
    return complex_tones(batch, N, alpha, 5, (0.1, 1.0), 0.1, seed)


def large_r32(batch=8, N=1 << 22, alpha=16, seed=4):
    return real_tones(batch, N, alpha, 20, (1e-4, 1.0), 1e-3, seed, dtype=np.float32,
                      log_amp=True, chunk=1)


RAGGED_ALPHAS = (2.0, 3.0, 4.0, 8.0, 2.5)


def ragged_shapes(count=10000, seed=5, e_lo=8, e_hi=16):
    """(N, alpha) per signal: N = 2^e, e ~ U{e_lo..e_hi}; alpha ~ U{2,3,4,8,2.5}."""
    rng = _rng(seed)
    e = rng.integers(e_lo, e_hi + 1, size=count)
    a = np.asarray(RAGGED_ALPHAS)[rng.integers(0, len(RAGGED_ALPHAS), size=count)]
    return (1 << e).astype(np.int64), a


def ragged_r32(count=10000, seed=5, e_lo=8, e_hi=16):
    """Packed ragged batch: returns (x_packed fp32, Ns, alphas, in_offsets)."""
    Ns, alphas = ragged_shapes(count, seed, e_lo, e_hi)
    offs = np.zeros(count + 1, dtype=np.int64)
    offs[1:] = np.cumsum(Ns)
    x = np.empty(int(offs[-1]), dtype=np.float32)
    rng = _rng(seed + 1000)
    for i in range(count):
        N = int(Ns[i])
        sub_seed = int(rng.integers(0, 2**62))
        xi, _ = real_tones(1, N, float(alphas[i]), 5, (0.1, 1.0), 0.2, sub_seed)
        x[offs[i]:offs[i + 1]] = xi[0]
    return x, Ns, alphas, offs
