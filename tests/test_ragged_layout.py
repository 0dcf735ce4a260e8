"""Host logic of the ragged queue form (no GPU): the tile list adfft_ragged_queue_layout
returns for the 10000-signal mix and for small mixes, against an independent statement of
its rules — every signal transformed exactly once, fft tiles covering each split signal's
residues and unpack tiles its leader bins exactly once, every unpack tile after all fft
tiles of its signal (the waits point only backwards in the queue, so the persistent kernel
cannot deadlock) and, where the queue continues, at least `lag` tiles after them."""
import math

import numpy as np
import pytest

from paper_2403_16665_gb300 import adfft, signals

TILE_POINTS = 4096      # complex points of U one tile holds
LEADERS = 8192          # leader bins of one unpack tile
MAX_GROUP = 64          # signals of one whole tile


def _lib():
    try:
        adfft.load()
    except RuntimeError as e:
        pytest.skip(str(e))


def geometry(N, M, real):
    """(Nc, Mc, Np, P, leaders) of a class, stated from the fold rule of Sec. 3: the
    largest power-of-two divisor of gcd(Mc, Nc), at most one tile."""
    Nc, Mc = (N // 2, M // 2) if real else (N, M)
    g = math.gcd(Mc, Nc)
    Np = min(g & -g, TILE_POINTS)
    jt = Mc // 2 + 1 if real else Mc
    return Nc, Mc, Np, Mc // Np, jt


def check_layout(Ns, alphas, real, lag):
    tiles, whole = adfft.ragged_queue_layout(Ns, alphas, adfft.R32 if real else adfft.C64, lag)
    Ms = np.rint(np.asarray(alphas) * np.asarray(Ns)).astype(np.int64)
    keys = sorted(set(zip(np.asarray(Ns).tolist(), Ms.tolist())))
    cls_of_key = {k: i for i, k in enumerate(keys)}
    geo = {k: geometry(k[0], k[1], real) for k in keys}
    n = len(Ns)
    split = np.array([geo[(int(Ns[s]), int(Ms[s]))][3] * geo[(int(Ns[s]), int(Ms[s]))][2] > TILE_POINTS
                      for s in range(n)])
    kind = tiles[:, 0]
    # every tile's class is its signal's (N, M) class
    for t in tiles[kind != 0]:
        assert t[1] == cls_of_key[(int(Ns[t[2]]), int(Ms[t[2]]))]
    # whole tiles: the unsplit signals, each once, groups of one class within one tile's points
    seen = np.zeros(n, dtype=np.int64)
    for t in tiles[kind == 0]:
        members = whole[t[2]:t[2] + t[4]]
        assert 1 <= t[4] <= MAX_GROUP
        ks = {(int(Ns[s]), int(Ms[s])) for s in members}
        assert len(ks) == 1 and cls_of_key[ks.pop()] == t[1]
        Mc = geo[(int(Ns[members[0]]), int(Ms[members[0]]))][1]
        assert t[4] == 1 or t[4] * Mc <= TILE_POINTS
        seen[members] += 1
    assert (seen[~split] == 1).all() and (seen[split] == 0).all()
    # whole tiles come last
    if (kind == 0).any() and (kind != 0).any():
        assert np.nonzero(kind == 0)[0].min() > np.nonzero(kind != 0)[0].max()
    # split signals: residues and leaders covered exactly once, unpack after fft (+ lag)
    fft_idx = {}
    unp_idx = {}
    for i, t in enumerate(tiles):
        if t[0] == 1:
            fft_idx.setdefault(int(t[2]), []).append(i)
        elif t[0] == 2:
            unp_idx.setdefault(int(t[2]), []).append(i)
    assert set(fft_idx) == set(np.nonzero(split)[0].tolist()) == set(unp_idx)
    fft_positions = np.nonzero(kind == 1)[0]
    for s in fft_idx:
        Nc, Mc, Np, P, jt = geo[(int(Ns[s]), int(Ms[s]))]
        res = np.zeros(P, dtype=np.int64)
        for i in fft_idx[s]:
            r0, cnt = tiles[i, 3], tiles[i, 4]
            assert 1 <= cnt <= TILE_POINTS // Np
            res[r0:r0 + cnt] += 1
        assert (res == 1).all()
        lead = np.zeros(jt, dtype=np.int64)
        for i in unp_idx[s]:
            j0, j1 = tiles[i, 3], tiles[i, 4]
            assert 0 < j1 - j0 <= LEADERS
            lead[j0:j1] += 1
        assert (lead == 1).all()
        last_fft, first_unp = max(fft_idx[s]), min(unp_idx[s])
        assert first_unp > last_fft
        if (fft_positions > first_unp).any():
            assert first_unp - (last_fft + 1) >= lag
    # split signals enter the queue largest M first
    first_fft = sorted((min(v), int(Ms[s])) for s, v in fft_idx.items())
    assert all(a[1] >= b[1] for a, b in zip(first_fft, first_fft[1:]))
    return tiles, whole


def test_layout_of_the_10000_signal_mix():
    _lib()
    Ns, alphas = signals.ragged_shapes(10000)
    tiles, whole = check_layout(Ns, alphas, True, 608)
    assert len(whole) > 0 and (tiles[:, 0] == 1).any()


@pytest.mark.parametrize("lag", [0, 1, 37, 100000])
def test_layout_lag_rule(lag):
    _lib()
    Ns, alphas = signals.ragged_shapes(300, seed=11)
    check_layout(Ns, alphas, True, lag)


def test_layout_complex_mix():
    _lib()
    rng = np.random.default_rng(3)
    Ns = [int(2 ** e) for e in rng.integers(8, 17, size=40)] + [65536, 256]
    alphas = list(rng.choice([2.0, 3.0, 4.0, 8.0, 2.5], size=40)) + [8.0, 2.0]
    check_layout(Ns, alphas, False, 16)


def test_layout_empty_and_single():
    _lib()
    tiles, whole = adfft.ragged_queue_layout([], [], adfft.R32, 8)
    assert tiles.shape == (0, 5) and whole.size == 0
    tiles, whole = adfft.ragged_queue_layout([256], [2.0], adfft.R32, 8)
    assert tiles.tolist() == [[0, 0, 0, 0, 1]] and whole.tolist() == [0]


def test_layout_refused_where_the_queue_cannot_serve():
    _lib()
    with pytest.raises(adfft.AdfftError):
        adfft.ragged_queue_layout([1000, 2000], [2.5, 2.5], adfft.C64, 8)   # fold of more than 64 blocks
    with pytest.raises(adfft.AdfftError):
        adfft.ragged_queue_layout([1001], [2.0], adfft.R32, 8)              # odd N, real: not packed
    with pytest.raises(adfft.AdfftError):
        adfft.ragged_queue_layout([256], [0.0], adfft.R32, 8)               # alpha must be > 0
