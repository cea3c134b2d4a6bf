"""The oracle's local-energy model (not gpu): the nonlinear short-range model
of Sec. 3 (qSRO), read as E = sum_i sum_m sum_s T_m[s_i][s][c_{i,m,s}], a
trial's energy change recomputed over the local energies of every site of the
interaction zone.  Pinned against: the brute-force local energy of
tests/bruteforce.py (distances over periodic images, no shared tables); the
EPI model, which is the linear table T = c V / 2 (energies, energy changes and
whole trajectories equal the EPI oracle's on the same link cells); exact
energy changes against full recomputation; conservation and the temperature
limits; the canonical distribution by enumeration; and the link-cell rule
(cell order irrelevant at the local model's L, relevant one below it)."""
import itertools
import math

import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs
from tests import bruteforce as bf
from tests.test_oracle_boltzmann import _compare, _exact_levels


def _table(kind, M, K, seed, scale=0.02):
    """A nonlinear table: per (shell, centre, neighbour species) a random
    function of the count (q units)."""
    import oracle
    zt = oracle.local_width(kind, M)
    rng = np.random.default_rng(seed)
    return np.round(rng.normal(0.0, scale, (M, K, K, zt)) * 2.0 ** 32).astype(np.int64)


def _linear_table(V, zt):
    M, K, _ = V.shape
    c = np.arange(zt, dtype=np.int64)
    return (V[:, :, :, None] // 2) * c[None, None, None, :]


def _even_epi(M, K, seed):
    V = inputs.epi_table(M, K, 0.03, seed)
    return (V // 2) * 2


CASES = [(0, (3, 4, 5), 3, 3), (1, (3, 3, 4), 3, 2), (0, (2, 2, 3), 4, 2), (1, (2, 3, 2), 3, 3),
         (0, (6, 6, 7), 5, 3), (1, (3, 4, 3), 8, 2)]


@pytest.mark.parametrize("kind,n,K,M", CASES)
def test_local_energy_equals_brute_force(orc, kind, n, K, M):
    T = _table(kind, M, K, seed=1)
    occ = inputs.initial_occupancy(kind, n, K, seed=2)
    d = orc.Desc(kind, n, K, M)
    assert orc.local_energy(d, T, occ) == bf.local_energies(kind, n, T, occ[None, :])[0]


@pytest.mark.parametrize("kind,n,K,M", CASES)
def test_linear_table_is_the_epi_model(orc, kind, n, K, M):
    V = _even_epi(M, K, seed=3)
    T = _linear_table(V, orc.local_width(kind, M))
    d = orc.Desc(kind, n, K, M)
    rng = np.random.default_rng(4)
    occ = inputs.initial_occupancy(kind, n, K, seed=5)
    assert orc.local_energy(d, T, occ) == orc.energy(d, V, occ)
    N = occ.size
    for _ in range(60):
        i, j = (int(v) for v in rng.integers(0, N, 2))
        assert orc.local_delta_e(d, T, occ, i, j) == orc.delta_e(d, V, occ, i, j)


@pytest.mark.parametrize("kind,n,K,M", CASES)
def test_delta_e_is_the_full_energy_difference(orc, kind, n, K, M):
    T = _table(kind, M, K, seed=6)
    d = orc.Desc(kind, n, K, M)
    rng = np.random.default_rng(7)
    occ = inputs.initial_occupancy(kind, n, K, seed=8)
    E0 = orc.local_energy(d, T, occ)
    N = occ.size
    for _ in range(40):
        i, j = (int(v) for v in rng.integers(0, N, 2))
        o = occ.copy()
        o[i], o[j] = o[j], o[i]
        assert orc.local_delta_e(d, T, occ, i, j) == orc.local_energy(d, T, o) - E0


def test_linear_table_sweeps_follow_the_epi_trajectory(orc):
    """Same link cells (the EPI run given min_cell = the local model's L):
    the two models' trajectories coincide bit for bit."""
    for kind, n, K, M in [(0, (12, 9, 10), 4, 3), (1, (8, 7, 9), 3, 2)]:
        V = _even_epi(M, K, seed=9)
        T = _linear_table(V, orc.local_width(kind, M))
        dl = orc.Desc(kind, n, K, M, seed=21)
        L, _ = orc.local_layout(dl)
        de = orc.Desc(kind, n, K, M, seed=21, min_cell=L)
        occ = inputs.initial_occupancy(kind, n, K, seed=10)
        a, sa = orc.local_sweeps(dl, T, occ, 0, 3, 1500.0, 700.0)
        b, sb = orc.sweeps(de, V, occ, 0, 3, 1500.0, 700.0)
        assert np.array_equal(a, b) and np.array_equal(sa, sb)


@pytest.mark.parametrize("kind,n,K,M", [(0, (7, 6, 8), 4, 3), (1, (6, 6, 7), 3, 3)])
def test_sweeps_conserve_and_track_the_energy(orc, kind, n, K, M):
    T = _table(kind, M, K, seed=11)
    d = orc.Desc(kind, n, K, M, seed=12)
    occ = inputs.initial_occupancy(kind, n, K, seed=13)
    E0 = orc.local_energy(d, T, occ)
    o, st = orc.local_sweeps(d, T, occ, 0, 4, 900.0)
    assert np.array_equal(np.bincount(o, minlength=K), np.bincount(occ, minlength=K))
    assert orc.local_energy(d, T, o) == E0 + int(st["sum_dE"].sum())
    assert int(st["attempts"].sum()) == 4 * occ.size
    # beta = 0 accepts every unlike trial; T = 0 never raises the energy
    _, s_inf = orc.local_sweeps(d, T, o, 4, 2, float("inf"))
    assert np.array_equal(s_inf["accepted"], s_inf["unlike"])
    _, s_0 = orc.local_sweeps(d, T, o, 6, 3, 0.0)
    assert np.all(s_0["sum_dE"] <= 0)


def test_layout_is_set_by_the_doubled_reach(orc):
    """L = floor((1 + 2 h_R)/2) + 1: h_R = 2 half units for BCC shells 1-3
    and FCC shells 1-3, 1 for BCC shell 1 and FCC shells 1-2."""
    for kind, M, L in [(0, 3, 3), (1, 3, 3), (0, 1, 2), (1, 2, 3), (1, 1, 2)]:
        d = orc.Desc(kind, (12, 12, 12), 3, M)
        assert orc.local_layout(d)[0] == L, (kind, M)


@pytest.mark.parametrize("kind,n", [(0, (12, 12, 12)), (1, (12, 12, 12))])
def test_cell_order_is_irrelevant_and_a_smaller_cell_breaks_it(orc, kind, n):
    K, M = 3, 3
    T = _table(kind, M, K, seed=14, scale=0.05)
    d = orc.Desc(kind, n, K, M, seed=15)
    n_try = 4 if kind == 0 else 2
    occ = inputs.initial_occupancy(kind, n, K, seed=16)
    L, _ = orc.local_layout(d)
    a, _ = orc.local_sweeps(d, T, occ, 0, 2, 800.0)
    b, _ = orc.local_sweeps(d, T, occ, 0, 2, 800.0, shuffle_cells=True, shuffle_seed=3)
    assert np.array_equal(a, b)
    differs = False
    for s in range(n_try):
        a2, _ = orc.local_sweeps(d, T, occ, 0, 2, 800.0, L_override=L - 1)
        b2, _ = orc.local_sweeps(d, T, occ, 0, 2, 800.0, L_override=L - 1, shuffle_cells=True,
                                 shuffle_seed=s + 5)
        differs |= not np.array_equal(a2, b2)
    assert differs


def test_single_cell_boltzmann_nonlinear_table(orc):
    """BCC 2x2x2 conventional cells, 8 + 8 atoms (12,870 states), one
    sequential cell: the chain's energy levels follow exp(-beta E) with E the
    brute-force local energy of a nonlinear table."""
    kind, n, M = 0, (2, 2, 2), 2
    N = 16
    T = _table(kind, M, 2, seed=17, scale=0.01)
    states = np.array([[1 if i in c else 0 for i in range(N)]
                        for c in itertools.combinations(range(N), 8)], dtype=np.uint8)
    E = bf.local_energies(kind, n, T, states)
    Temp = 1500.0
    levels, p = _exact_levels(E, Temp)
    d = orc.Desc(kind, n, 2, M, seed=4, flags=orc.FLAG_SINGLE_CELL)
    occ = states[321].copy()
    E0 = orc.local_energy(d, T, occ)
    o, st = orc.local_sweeps(d, T, occ, 0, 60000, Temp)
    Et = E0 + np.cumsum(st["sum_dE"].astype(np.int64))
    assert Et[-1] == orc.local_energy(d, T, o)
    _compare(levels, p, Et[500:])


def test_synthetic_table_shape_and_zero_count(orc):
    """inputs.local_energy_table: [M][K][K][1 + max z_m], no energy at a zero
    count, and nonlinear in the count (a quadratic term on top of c V / 2)."""
    for kind in (0, 1):
        T = inputs.local_energy_table(kind, 3, 5, 0.02, seed=3)
        assert T.shape == (3, 5, 5, orc.local_width(kind, 3)) and T.dtype == np.int64
        assert np.all(T[..., 0] == 0)
        lin = T[..., 1:2] * np.arange(T.shape[3])[None, None, None, :]
        assert np.any(T != lin)


def test_single_cell_boltzmann_fcc_nonlinear_table(orc):
    """FCC 2x2x2 conventional cells, 4 minority atoms in 32 (35,960 states),
    one sequential cell, shells 1-2 with a nonlinear table: the chain's
    energy levels follow exp(-beta E) of the brute-force local energy."""
    kind, n, M = 1, (2, 2, 2), 2
    N = 32
    T = _table(kind, M, 2, seed=19, scale=0.01)
    states = np.array([[1 if i in c else 0 for i in range(N)]
                       for c in itertools.combinations(range(N), 4)], dtype=np.uint8)
    E = bf.local_energies(kind, n, T, states)
    Temp = 1200.0
    levels, p = _exact_levels(E, Temp)
    d = orc.Desc(kind, n, 2, M, seed=8, flags=orc.FLAG_SINGLE_CELL)
    occ = states[777].copy()
    E0 = orc.local_energy(d, T, occ)
    o, st = orc.local_sweeps(d, T, occ, 0, 20000, Temp)
    Et = E0 + np.cumsum(st["sum_dE"].astype(np.int64))
    assert Et[-1] == orc.local_energy(d, T, o)
    _compare(levels, p, Et[500:])
