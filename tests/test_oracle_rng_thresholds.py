"""Pins of the oracle's Philox4x32-10 and Metropolis threshold tables (not gpu).

Philox (the counter-based generator the method keys by seed, sweep, cell and
trial) is checked statistically here; its bit-exact agreement with an
independent implementation (curand's device Philox4x32-10) is a gpu test.
The threshold tables implement the Metropolis acceptance exp(-beta dE)
(Sec. 2.1, Eq. 3) and are checked against the closed form and libm.
"""
import math

import numpy as np
import pytest
from scipy import stats

from tests import bruteforce as bf


def _stream(orc, n, key=(7, 11), c2=3):
    out = np.zeros((n, 4), dtype=np.uint32)
    for i in range(n):
        out[i] = orc.philox((i, 0, c2, 0), key)
    return out


def test_philox_byte_uniformity(orc):
    w = _stream(orc, 4000).view(np.uint8).ravel()
    h = np.bincount(w, minlength=256)
    chi2, p = stats.chisquare(h)
    assert p > 1e-4


def test_philox_bit_balance_and_avalanche(orc):
    w = _stream(orc, 2000)
    bits = np.unpackbits(w.view(np.uint8)).reshape(len(w), -1)
    frac = bits.mean(0)
    assert np.all(np.abs(frac - 0.5) < 5 * 0.5 / math.sqrt(len(w)))
    # flipping one counter bit flips about half of the 128 output bits
    rng = np.random.default_rng(0)
    flips = []
    for _ in range(300):
        c = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
        k = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
        b = int(rng.integers(0, 128))
        c2 = c.copy()
        c2[b // 32] ^= np.uint32(1 << (b % 32))
        d = orc.philox(c, k) ^ orc.philox(c2, k)
        flips.append(int(np.unpackbits(d.view(np.uint8)).sum()))
    assert abs(np.mean(flips) - 64) < 2.0


def test_philox_key_and_counter_sensitivity(orc):
    a = orc.philox((0, 0, 0, 0), (0, 0))
    assert not np.all(a == 0)
    assert not np.array_equal(a, orc.philox((0, 0, 0, 0), (1, 0)))
    assert not np.array_equal(a, orc.philox((0, 0, 0, 0), (0, 1)))
    seen = {tuple(orc.philox((i, j, 0, 0), (5, 5))) for i in range(100) for j in range(20)}
    assert len(seen) == 2000


KB = bf.golden("constants.json")["k_B_eV_per_K"]
Q = 2.0 ** -32


@pytest.mark.parametrize("T", [3.0, 300.0, 600.0, 800.0, 1000.0, 1200.0, 1500.0, 1e5])
def test_threshold_tables(orc, T):
    tab, s, mode = orc.thresholds(T)
    assert mode == orc.MODE_NORMAL
    beta = 1.0 / (KB * T)
    # s: largest integer >= 0 with beta q 2^s <= 2^-20
    assert beta * Q * 2.0 ** s <= 2.0 ** -20 or s == 0
    assert beta * Q * 2.0 ** (s + 1) > 2.0 ** -20
    assert tab[0, 0] == 2 ** 32 - 1 and tab[1, 0] == 2 ** 32 - 1 and tab[2, 0] == 2 ** 32 - 1
    for l in range(3):
        assert np.all(np.diff(tab[l].astype(np.int64)) <= 0)
    # composed threshold vs the closed form at the bin's lower edge
    rng = np.random.default_rng(1)
    idx = np.concatenate([np.arange(2000), rng.integers(0, 2 ** 27, 20000)])
    a = tab[0, idx & 511].astype(object)
    b = tab[1, (idx >> 9) & 511].astype(object)
    c = tab[2, idx >> 18].astype(object)
    thr = np.array([((int(x) * int(y) >> 32) * int(z)) >> 32 for x, y, z in zip(a, b, c)],
                   dtype=np.float64)
    exact = 2.0 ** 32 * np.exp(-beta * Q * 2.0 ** s * idx.astype(np.float64))
    big = exact > 2.0 ** 20
    rel = np.abs(thr[big] - exact[big]) / exact[big]
    assert rel.max() <= 2.0 ** -19
    assert np.all(np.abs(thr[~big] - exact[~big]) <= 4.0)
    # lower-edge binning: the bin's width costs at most 2^-20 in relative terms
    assert beta * Q * 2.0 ** s <= 2.0 ** -20


def test_threshold_limits(orc):
    tab, s, mode = orc.thresholds(0.0)
    assert mode == orc.MODE_ZERO_T
    tab, s, mode = orc.thresholds(float("inf"))
    assert mode == orc.MODE_ACCEPT_ALL
    with pytest.raises(orc.OracleError):
        orc.thresholds(-1.0)
    with pytest.raises(orc.OracleError):
        orc.thresholds(float("nan"))
    # below ~2.83 K even s = 0 overshoots 2^-20: s stays 0
    tab, s, mode = orc.thresholds(1.0)
    assert s == 0 and mode == orc.MODE_NORMAL
