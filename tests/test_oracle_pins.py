"""Pins of the FP64 direct-sum oracle against what the paper and mathematics fix.

Each test names the passage it follows.  Together they are chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign of the exponent,
an index off by one, a transposed operand, a wrong scale) fails at least one.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import closed_form as cf

RNG = np.random.default_rng(12345)


def _rand(N, complex_=True, batch=None):
    shape = (N,) if batch is None else (batch, N)
    x = RNG.standard_normal(shape)
    if complex_:
        x = x + 1j * RNG.standard_normal(shape)
    return x


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("N,M,cplx", [(1, 1, False), (1, 5, True), (2, 8, True), (7, 7, False),
                                      (8, 20, True), (6, 4, True), (12, 30, False),
                                      (16, 40, True), (64, 256, False)])
def test_brute_force_extended_precision(N, M, cplx):
    """Eq. 7 evaluated term by term in 40-digit arithmetic with exact rational angles."""
    mp = pytest.importorskip("mpmath")
    x = _rand(N, cplx)
    S = 1.0 / N
    got = oracle.alpha_dft(x, M)
    with mp.workdps(40):
        for m in range(M):
            acc = mp.mpc(0)
            for n in range(N):
                fr = Fraction(m * n % M, M)              # exact phase in turns
                ang = -2 * mp.pi * fr.numerator / fr.denominator
                acc += mp.mpc(float(np.real(x[n])), float(np.imag(x[n]))) * mp.expj(ang)
            ref = complex(acc * S)
            assert abs(got[m] - ref) <= 1e-14 * max(1.0, abs(ref)), (m, got[m], ref)


# ---------------------------------------------------------------- alpha = 1
@pytest.mark.parametrize("N", [1, 2, 5, 16, 100, 1024])
def test_alpha_one_is_textbook_dft(N):
    """alpha = 1 reduces Eq. 7 to the standard DFT of Eq. 5 (times S = T/N of Eq. 2)."""
    x = _rand(N)
    got = oracle.alpha_dft(x, N)
    ref = np.fft.fft(x) / N
    assert _rel(got, ref) < 1e-14


# ---------------------------------------------------------------- zero padding
@pytest.mark.parametrize("N,M,cplx", [(64, 256, False), (100, 250, True), (1024, 4096, False),
                                      (8, 8 * 16, True), (512, 1920, True), (300, 301, False)])
def test_equals_zero_padded_dft(N, M, cplx):
    """alpha > 1 equals appending (alpha-1)N zeros before a length-alpha N DFT (Sec. 2)."""
    x = _rand(N, cplx)
    got = oracle.alpha_dft(x, M)
    ref = np.fft.fft(x, n=M) / N
    assert _rel(got, ref) < 1e-14
    assert np.max(np.abs(got - ref)) < 1e-14 * max(1.0, np.max(np.abs(ref)))


# ---------------------------------------------------------------- integer / rational alpha
@pytest.mark.parametrize("N,alpha", [(32, 2), (50, 3), (64, 8), (17, 4)])
def test_integer_alpha_every_alpha_th_bin_is_plain_dft(N, alpha):
    """W_{alpha N}^{alpha k n} = W_N^{kn} (Eq. 9, second property applied log2 alpha times)."""
    x = _rand(N)
    dense = oracle.alpha_dft(x, alpha * N)
    plain = oracle.alpha_dft(x, N)
    assert _rel(dense[::alpha], plain) < 1e-14


@pytest.mark.parametrize("N,p,q", [(8, 5, 2), (16, 15, 4), (12, 2, 3), (20, 7, 5)])
def test_rational_alpha_is_subsampled_integer_alpha(N, p, q):
    """alpha = p/q: X^{(p/q)}_m = X^{(p)}_{q m} since W_{pN/q}^{mn} = W_{pN}^{qmn} (Eq. 7)."""
    x = _rand(N)
    M = p * N // q
    assert M * q == p * N
    got = oracle.alpha_dft(x, M)
    fine = oracle.alpha_dft(x, p * N)
    assert _rel(got, fine[::q][:M]) < 1e-14


# ---------------------------------------------------------------- tones
@pytest.mark.parametrize("N,alpha", [(64, 4), (1024, 4), (128, 2.5), (256, 1), (100, 3)])
def test_off_grid_tone_closed_form_every_bin(N, alpha):
    """A tone nu cycles over T: Eq. 7 is a geometric series, known at every bin."""
    M = int(round(alpha * N))
    # float64 closed form: its phase pi*delta*N carries an error of order pi*N*eps
    tol = max(1e-13, 2 * np.pi * N * 2.2e-16)
    for nu, A, phi in [(3.3, 1.7, 0.4), (N / 2 - 0.61, 0.5, 2.0), (0.17, 2.0, -1.0)]:
        n = np.arange(N)
        x = A * np.exp(1j * (2 * np.pi * nu * n / N + phi))
        got = oracle.alpha_dft(x, M)
        ref = cf.tone_spectrum(N, M, nu, A, phi)
        assert np.max(np.abs(got - ref)) < tol * A, (nu,)
        xr = A * np.cos(2 * np.pi * nu * n / N + phi)
        got_r = oracle.alpha_dft(xr, M)
        ref_r = cf.cosine_spectrum(N, M, nu, A, phi)
        assert np.max(np.abs(got_r - ref_r)) < tol * A


@pytest.mark.parametrize("N,alpha,j", [(64, 4, 9), (32, 8, 5), (128, 2, 7), (16, 1, 3)])
def test_tone_on_fine_grid(N, alpha, j):
    """Tone at frequency j/(alpha T) (Eq. 6): X_j = T*A; bins m = j mod alpha, m != j, are 0.

    For alpha = 1 this is the single nonzero bin of value T*A; for alpha > 1 the
    remaining bins carry the Dirichlet leakage given by the closed form.
    """
    M = alpha * N
    A, T = 1.3, 1.0
    n = np.arange(N)
    x = A * np.exp(2j * np.pi * (j / alpha) * n / N)
    X = oracle.alpha_dft(x, M)
    assert abs(X[j] - T * A) < 1e-14
    same = np.arange(j % alpha, M, alpha)
    same = same[same != j]
    assert np.max(np.abs(X[same]), initial=0.0) < 1e-14
    if alpha == 1:
        others = np.delete(np.arange(M), j)
        assert np.max(np.abs(X[others])) < 1e-14
    ref = cf.tone_spectrum(N, M, j / alpha, A)
    assert np.max(np.abs(X - ref)) < 1e-13


# ---------------------------------------------------------------- structure
def test_linearity():
    N, M = 96, 240
    x, y = _rand(N), _rand(N)
    a, b = 0.7 - 0.2j, -1.9 + 0.5j
    lhs = oracle.alpha_dft(a * x + b * y, M)
    rhs = a * oracle.alpha_dft(x, M) + b * oracle.alpha_dft(y, M)
    assert _rel(lhs, rhs) < 1e-14


@pytest.mark.parametrize("N,M", [(64, 64), (64, 256), (80, 200), (33, 99)])
def test_parseval_from_alpha_orthogonality(N, M):
    """Eq. 8: columns of the N x M matrix are orthogonal when M >= N, so
    sum_m |X_m|^2 = S^2 M sum_n |x_n|^2."""
    x = _rand(N)
    X = oracle.alpha_dft(x, M)
    S = 1.0 / N
    assert abs(np.sum(np.abs(X) ** 2) - S * S * M * np.sum(np.abs(x) ** 2)) < 1e-12 * np.sum(np.abs(X) ** 2)


@pytest.mark.parametrize("N,M", [(64, 256), (50, 125), (31, 62)])
def test_real_input_hermitian(N, M):
    x = _rand(N, complex_=False)
    X = oracle.alpha_dft(x, M)
    m = np.arange(1, M)
    assert np.max(np.abs(X[M - m] - np.conj(X[m]))) < 1e-15 * np.max(np.abs(X)) + 1e-16
    assert abs(X[0].imag) < 1e-15


def test_scale_and_sampled_bins():
    N, M = 40, 100
    x = _rand(N)
    full = oracle.alpha_dft(x, M, S=1.0)
    bins = np.array([99, 0, 37, 37, 50])
    part = oracle.alpha_dft(x, M, S=1.0, bins=bins)
    assert np.array_equal(part, full[bins])
    assert _rel(oracle.alpha_dft(x, M), full / N) < 1e-15
    with pytest.raises(ValueError):
        oracle.alpha_dft(x, M, bins=[M])


def test_batch_rows_are_independent():
    x = _rand(24, batch=3)
    X = oracle.alpha_dft(x, 72)
    for b in range(3):
        assert np.array_equal(X[b], oracle.alpha_dft(x[b], 72))


# ---------------------------------------------------------------- adjoint / inverse
@pytest.mark.parametrize("N,M", [(16, 64), (30, 75), (64, 32)])
def test_adjoint_dot_product(N, M):
    """<A x, g> = <x, A^H g> for the matrix of Eq. 7 (catches a transposed operand)."""
    x, g = _rand(N), _rand(M)
    Ax = oracle.alpha_dft(x, M)
    Ahg = oracle.alpha_dft_adjoint(g, N)
    lhs = np.vdot(g, Ax)
    rhs = np.vdot(Ahg, x)
    assert abs(lhs - rhs) < 1e-13 * max(1.0, abs(lhs))


@pytest.mark.parametrize("N,alpha", [(16, 4), (40, 2.5), (64, 1)])
def test_inverse_of_eq7_recovers_signal(N, alpha):
    """Second line of Eq. 7: x_n = (1/(alpha N)) sum_m exp(+2 pi i mn/(alpha N)) X_m (S = 1)."""
    M = int(round(alpha * N))
    x = _rand(N)
    X = oracle.alpha_dft(x, M, S=1.0)
    back = oracle.alpha_dft_adjoint(X, N, S=1.0) / M
    assert _rel(back, x) < 1e-14


def test_adjoint_against_direct_matrix():
    N, M = 12, 30
    n, m = np.arange(N), np.arange(M)
    A = np.exp(-2j * np.pi * np.outer(m, n) / M) / N
    g = _rand(M)
    assert _rel(oracle.alpha_dft_adjoint(g, N), A.conj().T @ g) < 1e-14
    gr = oracle.alpha_dft_adjoint(g, N, real_input=True)
    assert _rel(gr, np.real(A.conj().T @ g)) < 1e-14


@pytest.mark.parametrize("N,M", [(12, 30), (64, 256), (50, 20)])
def test_sampled_adjoint_equals_full_adjoint(N, M):
    """The sampled-output adjoint evaluates the same sums as the full adjoint at the chosen
    samples (bit for bit), in the order given, for one and several signals; and, independently,
    the explicit conjugate-transposed matrix of Eq. 7 at those samples."""
    rng = np.random.default_rng(N + M)
    g = _rand(M) if N % 2 else np.stack([_rand(M) for _ in range(3)])
    samples = rng.permutation(N)[: max(1, N // 3)]
    full = oracle.alpha_dft_adjoint(g, N)
    part = oracle.alpha_dft_adjoint(g, N, samples=samples)
    assert np.array_equal(part, full[..., samples])
    A = np.exp(-2j * np.pi * np.outer(np.arange(M), samples) / M) / N
    assert _rel(part, (A.conj().T @ np.atleast_2d(g).T).T.reshape(part.shape)) < 1e-13
    assert np.array_equal(oracle.alpha_dft_adjoint(g, N, real_input=True, samples=samples),
                          np.real(full[..., samples]))
    with pytest.raises(ValueError):
        oracle.alpha_dft_adjoint(g, N, samples=[N])


@pytest.mark.parametrize("N,M", [(12, 8), (40, 10), (9, 6)])
def test_alpha_below_one_aliasing(N, M):
    """Sec. 2, alpha < 1: reconstruction through Eq. 8 folds the signal,
    x'_n = sum_k x_{n + k alpha N} over 0 <= n + k alpha N < N."""
    x = _rand(N)
    X = oracle.alpha_dft(x, M, S=1.0)
    back = oracle.alpha_dft_adjoint(X, N, S=1.0) / M
    ref = np.array([sum(x[l] for l in range(N) if (l - n) % M == 0) for n in range(N)])
    assert _rel(back, ref) < 1e-14


# ---------------------------------------------------------------- golden (paper's example)
def test_golden_sin_pi_t():
    """The paper's worked example, sin(pi t) on [0, 1] (Sec. 2, Figs. 1-2), against its
    closed form stored in tests/golden/sin_pi_t.txt."""
    path = os.path.join(os.path.dirname(__file__), "golden", "sin_pi_t.txt")
    rows = np.loadtxt(path, comments="#")
    for (N, M) in sorted({(int(r[0]), int(r[1])) for r in rows}):
        sel = rows[(rows[:, 0] == N) & (rows[:, 1] == M)]
        ref = sel[:, 3] + 1j * sel[:, 4]
        x = np.sin(np.pi * np.arange(N) / N)
        got = oracle.alpha_dft(x, M)
        assert np.max(np.abs(got - ref)) < 2e-16 * N, (N, M)


def test_output_bins_rule():
    assert oracle.output_bins(8192, 2.5) == 20480
    assert oracle.output_bins(8192, 3.75) == 30720
    with pytest.raises(ValueError):
        oracle.output_bins(10, 0.33)
