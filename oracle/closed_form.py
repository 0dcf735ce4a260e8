"""Closed-form alpha-DFT spectra of pure tones (test infrastructure only).

These are the analytic values the direct-sum oracle is pinned against; they
share no arithmetic with ``adfft_oracle.c``.

For a complex tone x_n = A * exp(i*(2*pi*nu*n/N + phi)) (nu cycles over the
record length T, sampled at t_n = nT/N as in Eq. 3), Eq. 7 with scale S is a
geometric series:

    X_m = S * A * e^{i phi} * sum_{n<N} z^n,   z = exp(2 pi i * delta),
    delta = nu/N - m/M = (alpha*nu - m)/M,

    sum_{n<N} z^n = exp(i pi delta (N-1)) * sin(pi delta N) / sin(pi delta)
                  (= N when delta is an integer).

A real cosine A cos(2 pi nu n/N + phi) is the sum of the tones (A/2, nu, phi)
and (A/2, -nu, -phi).  The paper's worked example x(t) = sin(pi t) on [0, 1]
(Sec. 2, Figs. 1 and 2) is the real cosine with nu = 1/2, phi = -pi/2.
"""
from __future__ import annotations

import numpy as np


def _dirichlet_np(delta, N):
    """sum_{n<N} exp(2 pi i delta n) in float64, stable near integer delta."""
    delta = np.asarray(delta, dtype=np.float64)
    frac = delta - np.round(delta)               # the sum only depends on delta mod 1
    out = np.empty(frac.shape, dtype=np.complex128)
    small = np.abs(frac) < 1e-15
    f = frac[~small]
    out[~small] = np.exp(1j * np.pi * f * (N - 1)) * np.sin(np.pi * f * N) / np.sin(np.pi * f)
    # delta integer (or indistinguishable from it): every term is 1
    out[small] = N * np.exp(1j * np.pi * frac[small] * (N - 1))
    return out


def tone_spectrum(N, M, nu, A=1.0, phi=0.0, S=None, bins=None):
    """Eq. 7 of a complex tone A exp(i(2 pi nu n/N + phi)) at the given bins (float64).

    nu is given as a float; for exact on-grid checks pass nu = j*N/M exactly
    representable (e.g. M a power of two).
    """
    S = 1.0 / N if S is None else S
    m = np.arange(M) if bins is None else np.asarray(bins)
    delta = nu / N - m / M
    return S * A * np.exp(1j * phi) * _dirichlet_np(delta, N)


def cosine_spectrum(N, M, nu, A=1.0, phi=0.0, S=None, bins=None):
    """Eq. 7 of a real cosine A cos(2 pi nu n/N + phi) (sum of two tones)."""
    return (tone_spectrum(N, M, nu, A / 2, phi, S, bins)
            + tone_spectrum(N, M, -nu, A / 2, -phi, S, bins))


def tone_spectrum_mp(N, M, nu_num, nu_den, A="1", phi_over_pi="0", S=None, bins=None, dps=40):
    """Same closed form in mpmath with an exact rational frequency nu = nu_num/nu_den.

    The phase offset is phi = pi * phi_over_pi (phi_over_pi a decimal string or
    rational).  Returns a list of (re, im) mpmath numbers.
    """
    import mpmath as mp
    with mp.workdps(dps):
        from fractions import Fraction
        nu = Fraction(nu_num, nu_den)
        Sm = mp.mpf(1) / N if S is None else mp.mpf(S)
        Am = mp.mpf(A)
        ph = mp.pi * mp.mpf(Fraction(phi_over_pi).numerator) / Fraction(phi_over_pi).denominator
        ms = range(M) if bins is None else bins
        out = []
        for m in ms:
            delta = nu / N - Fraction(m, M)       # exact rational
            frac = delta - round(delta)
            if frac == 0:
                s = mp.mpf(N)
                val = Sm * Am * mp.expj(ph) * s
            else:
                d = mp.mpf(frac.numerator) / frac.denominator
                s = mp.expj(mp.pi * d * (N - 1)) * mp.sin(mp.pi * d * N) / mp.sin(mp.pi * d)
                val = Sm * Am * mp.expj(ph) * s
            out.append((mp.re(val), mp.im(val)))
        return out


def sin_pi_t_spectrum_mp(N, M, dps=40):
    """Closed form of Eq. 7 (S = T/N, T = 1) for x_n = sin(pi n/N), the paper's example.

    sin(pi n/N) = cos(2 pi (1/2) n/N - pi/2) = (1/2i)(e^{i pi n/N} - e^{-i pi n/N}).
    """
    import mpmath as mp
    with mp.workdps(dps):
        a = tone_spectrum_mp(N, M, 1, 2, A="0.5", phi_over_pi="-1/2", dps=dps)
        b = tone_spectrum_mp(N, M, -1, 2, A="0.5", phi_over_pi="1/2", dps=dps)
        return [(ar + br, ai + bi) for (ar, ai), (br, bi) in zip(a, b)]
