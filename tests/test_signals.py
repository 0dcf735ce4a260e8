"""CPU checks of the seeded input generators: the stated recipe (shapes, dtypes,
tone count, amplitude ranges, off-grid frequencies, noise level) and determinism."""
import numpy as np
import pytest

from paper_2403_16665_gb300 import signals


def _residual(x, prm, N, complex_=False):
    n = np.arange(N, dtype=np.float64)
    acc = np.zeros_like(x, dtype=np.complex128 if complex_ else np.float64)
    for t in range(prm["nu"].shape[1]):
        ph = (2 * np.pi / N) * prm["nu"][:, t, None] * n[None, :] + prm["phi"][:, t, None]
        acc += prm["A"][:, t, None] * (np.exp(1j * ph) if complex_ else np.cos(ph))
    return x.astype(acc.dtype) - acc


def test_deterministic_per_seed_and_different_across_seeds():
    a, pa = signals.batch_r32(batch=3, N=256, seed=2)
    b, pb = signals.batch_r32(batch=3, N=256, seed=2)
    c, _ = signals.batch_r32(batch=3, N=256, seed=3)
    assert np.array_equal(a, b) and np.array_equal(pa["nu"], pb["nu"])
    assert not np.array_equal(a, c)


@pytest.mark.parametrize("alpha", [8, 2.5, 3.75, 16])
def test_frequencies_are_off_both_grids(alpha):
    _, p = signals.real_tones(64, 512, alpha, 5, (0.1, 1.0), 0.2, seed=11)
    nu = p["nu"]
    assert np.all((nu >= 0) & (nu < 256))
    frac = np.abs(alpha * nu - np.round(alpha * nu))
    assert frac.min() >= 0.05                  # off the 1/(alpha T) grid
    if float(alpha).is_integer():              # the 1/T grid is a subset of it
        assert np.abs(nu - np.round(nu)).min() >= 0.05 / alpha


def test_batch_r32_recipe():
    x, p = signals.batch_r32(batch=16, N=1024, alpha=8, seed=2)
    assert x.shape == (16, 1024) and x.dtype == np.float32
    assert p["nu"].shape == (16, 5)
    assert p["A"].min() >= 0.1 and p["A"].max() <= 1.0
    r = _residual(x, p, 1024)
    assert abs(r.std() - 0.2) < 0.01          # white noise, sigma = 0.2 (fp32 rounding is far below)


def test_batch_c64_recipe():
    x, p = signals.batch_c64(batch=8, N=2048, alpha=2.5, seed=3)
    assert x.shape == (8, 2048) and x.dtype == np.complex64
    assert np.all((p["nu"] >= 0) & (p["nu"] < 2048))
    r = _residual(x, p, 2048, complex_=True)
    assert abs(np.sqrt(np.mean(np.abs(r) ** 2)) - 0.1) < 0.005   # E|w|^2 = 0.1^2


def test_large_r32_recipe_small_instance():
    x, p = signals.large_r32(batch=2, N=1 << 12, alpha=16, seed=4)
    assert x.shape == (2, 4096) and x.dtype == np.float32
    assert p["nu"].shape == (2, 20)
    assert p["A"].min() >= 1e-4 and p["A"].max() <= 1.0
    assert p["A"].min() < 1e-2                 # log-uniform: several decades are drawn
    r = _residual(x, p, 4096)
    assert abs(r.std() - 1e-3) < 1e-4


def test_ragged_packing_and_shapes():
    x, Ns, alphas, offs = signals.ragged_r32(count=40, seed=5, e_lo=4, e_hi=9)
    assert offs[0] == 0 and offs[-1] == x.size and np.array_equal(np.diff(offs), Ns)
    assert set(np.log2(Ns).astype(int)) <= set(range(4, 10))
    assert set(alphas.tolist()) <= set(signals.RAGGED_ALPHAS)
    assert np.all(np.abs(alphas * Ns - np.round(alphas * Ns)) == 0)   # M = alpha N is an integer
    Ns2, a2 = signals.ragged_shapes(count=40, seed=5, e_lo=4, e_hi=9)
    assert np.array_equal(Ns, Ns2) and np.array_equal(alphas, a2)
