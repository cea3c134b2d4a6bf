"""The oracle's chain samples the canonical distribution (not gpu).

P(sigma) ~ exp(-beta H(sigma)) (Sec. 2.1, Eq. 1) is computed exactly by
enumerating every configuration of tiny two-species lattices with the
brute-force energies of tests/bruteforce.py; the oracle's chain (Metropolis
swaps, Eq. 3, over link-cell sweeps, Sec. 2.2) must reproduce the occupation
of every energy level within 5 batch-means standard errors.  One case is a
single sequential cell, two use a real checkerboard (several cells per colour
and a random origin every sweep).
"""
import itertools
import math

import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs
from tests import bruteforce as bf

KB = bf.golden("constants.json")["k_B_eV_per_K"]
Q = 2.0 ** 32


def _exact_levels(energies_q, T):
    beta_q = 1.0 / (KB * T) / Q
    E = np.array([int(e) for e in energies_q], dtype=object)
    levels = sorted(set(E))
    g = np.array([int((E == l).sum()) for l in levels], dtype=np.float64)
    e = np.array([float(l) for l in levels])
    w = g * np.exp(-beta_q * (e - e.min()))
    return np.array(levels, dtype=object), w / w.sum()


def _chain_levels(orc, d, V, occ, T, n_sweeps, burn=500):
    E0 = orc.energy(d, V, occ)
    occ2, st = orc.sweeps(d, V, occ, 0, n_sweeps, T)
    Et = E0 + np.cumsum(st["sum_dE"].astype(np.int64))
    assert Et[-1] == orc.energy(d, V, occ2)
    return Et[burn:]


def _compare(levels, p_exact, Et, n_batches=40, zmax=5.0):
    lv = np.array([int(l) for l in levels], dtype=np.int64)
    idx = np.searchsorted(lv, Et)
    assert np.all(lv[idx] == Et), "chain visited an energy with no configuration"
    B = len(Et) // n_batches
    worst = 0.0
    for k, p in enumerate(p_exact):
        if p < 2e-3:
            continue
        ind = (idx[: B * n_batches] == k).reshape(n_batches, B).mean(1)
        se = ind.std(ddof=1) / math.sqrt(n_batches)
        z = abs(ind.mean() - p) / max(se, 1e-4)
        worst = max(worst, z)
    assert worst < zmax, worst
    return worst


def _binary_V(M, seed, sigma=0.04):
    return inputs.epi_table(M, 2, sigma, seed)


def test_single_cell_bcc16(orc):
    """BCC 2x2x2 conventional cells, 8 + 8 atoms (12,870 states), one cell."""
    n = (2, 2, 2)
    N = 16
    V = _binary_V(2, 31)
    states = np.array([[1 if i in c else 0 for i in range(N)]
                        for c in itertools.combinations(range(N), 8)], dtype=np.uint8)
    E = bf.binary_energies(0, n, V, states)
    T = 1500.0
    levels, p = _exact_levels(E, T)
    d = orc.Desc(0, n, 2, 2, seed=4, flags=orc.FLAG_SINGLE_CELL)
    occ = states[123].copy()
    Et = _chain_levels(orc, d, V, occ, T, 120000)
    _compare(levels, p, Et)


def test_single_cell_fcc32_four_minority(orc):
    """FCC 2x2x2 conventional cells, 4 minority atoms in 32 (35,960 states)."""
    n = (2, 2, 2)
    N = 32
    V = _binary_V(2, 7, sigma=0.05)
    states = np.zeros((math.comb(N, 4), N), dtype=np.uint8)
    for r, c in enumerate(itertools.combinations(range(N), 4)):
        states[r, list(c)] = 1
    E = bf.binary_energies(1, n, V, states)
    T = 1200.0
    levels, p = _exact_levels(E, T)
    d = orc.Desc(1, n, 2, 2, seed=9)
    L, m = orc.layout(d)
    assert m == (1, 1, 1)
    occ = states[0].copy()
    Et = _chain_levels(orc, d, V, occ, T, 60000)
    _compare(levels, p, Et)


def test_checkerboard_two_minority_bcc(orc):
    """BCC 8x8x8 (1024 sites, 4x4x4 cells, 8 cells per colour, random origin
    every sweep) with two minority atoms: 523,776 states whose energies fall
    into 'apart', 'first-shell pair' and 'second-shell pair'."""
    n = (8, 8, 8)
    kind = 0
    N = 1024
    vab = int(round(0.02 * Q))
    vbb1 = int(round(-0.12 * Q))
    vbb2 = int(round(-0.05 * Q))
    V = np.array([[[0, vab], [vab, vbb1]], [[0, vab], [vab, vbb2]]], dtype=np.int64)
    # exact: the energy of a configuration depends only on the pair's shell
    E_apart = bf.energy(kind, n, V, _two(N, 0, 300))
    probe = {}
    P = bf.positions(kind, n)
    for j in range(1, N):
        dv = P[j] - P[0]
        dv = (dv + 8) % 16 - 8
        d2 = int((dv * dv).sum())
        if d2 in (3, 4) and d2 not in probe:
            probe[d2] = bf.energy(kind, n, V, _two(N, 0, j))
    n1, n2 = N * 8 // 2, N * 6 // 2
    n_apart = N * (N - 1) // 2 - n1 - n2
    T = 1000.0
    levels, p = _exact_levels([E_apart] * 1 + [probe[3]] + [probe[4]], T)
    # replace unit degeneracies by the true counts
    g = {int(E_apart): n_apart, int(probe[3]): n1, int(probe[4]): n2}
    beta_q = 1.0 / (KB * T) / Q
    e = np.array([float(l) for l in levels])
    w = np.array([g[int(l)] for l in levels], dtype=np.float64) * np.exp(-beta_q * (e - e.min()))
    p = w / w.sum()
    d = orc.Desc(kind, n, 2, 2, seed=13)
    L, m = orc.layout(d)
    assert m == (4, 4, 4)
    Et = _chain_levels(orc, d, V, _two(N, 0, 500), T, 40000, burn=200)
    _compare(levels, p, Et)


def _two(N, i, j):
    occ = np.zeros(N, dtype=np.uint8)
    occ[i] = 1
    occ[j] = 1
    return occ


def test_checkerboard_fcc_three_minority_levels(orc):
    """FCC 4x4x4 (256 sites, 2x2x2 cells) with three minority atoms
    (2,763,520 states): exact levels from a full enumeration."""
    n = (4, 4, 4)
    kind = 1
    N = 256
    V = np.array([[[0, int(0.01 * Q)], [int(0.01 * Q), int(-0.1 * Q)]]], dtype=np.int64)
    mult = bf.multiplicity(kind, n, 1)[0]
    A = (mult > 0).astype(np.int64) * mult
    # energy relative to all-majority: for minority set S, the change is
    # sum over ordered pairs; with V00 = 0 it is
    #   1/2 [ sum_{i,j in S} A_ij V11 + 2 sum_{i in S, j notin S} A_ij V01 ]
    v01, v11 = int(V[0, 0, 1]), int(V[0, 1, 1])
    z = int(A[0].sum())
    Es = []
    for S in itertools.combinations(range(N), 3):
        inner = int(A[np.ix_(S, S)].sum())
        Es.append((inner * v11 + 2 * (3 * z - inner) * v01) // 2)
    T = 900.0
    levels, p = _exact_levels(Es, T)
    d = orc.Desc(kind, n, 2, 1, seed=21)
    L, m = orc.layout(d)
    assert m == (2, 2, 2)
    occ = np.zeros(N, dtype=np.uint8)
    occ[[0, 100, 200]] = 1
    E0 = orc.energy(d, V, occ)
    occ2, st = orc.sweeps(d, V, occ, 0, 40000, T)
    Et = E0 + np.cumsum(st["sum_dE"].astype(np.int64))[200:]
    _compare(levels, p, Et)
