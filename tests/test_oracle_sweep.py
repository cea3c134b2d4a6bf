"""Pins of the oracle's sweep (not gpu).

One MC step visits every site once (Sec. 2.1); link cells of one colour are
updated as non-interacting blocks (Sec. 2.2); acceptance is Metropolis
(Sec. 2.1, Eq. 3).  Checked here: exact species conservation, running energy
= full recompute, the beta = 0 / T = 0 / K = 1 limits, independence of the
order of same-colour cells (and that the check fails when cells are made too
small), and the textbook B2 ground state of an ordering binary BCC alloy.
"""
import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs

Q = 2.0 ** 32


def _setup(orc, kind, n, K, M, seed=0, sigma=0.03, flags=0, epi_seed=1):
    d = orc.Desc(kind, n, K, M, seed=seed, flags=flags)
    V = inputs.epi_table(M, K, sigma, seed=epi_seed)
    occ = inputs.initial_occupancy(kind, n, K, seed=seed + 17)
    return d, V, occ


@pytest.mark.parametrize("kind,n,K,M", [(0, (8, 8, 8), 4, 2), (1, (4, 6, 4), 5, 4),
                                        (0, (5, 7, 6), 3, 3), (1, (3, 3, 3), 6, 3),
                                        (0, (2, 2, 2), 2, 2)])
def test_conservation_and_running_energy(orc, kind, n, K, M):
    d, V, occ = _setup(orc, kind, n, K, M)
    E = orc.energy(d, V, occ)
    counts0 = np.bincount(occ, minlength=K)
    t = 0
    for chunk in range(4):
        occ, st = orc.sweeps(d, V, occ, t, 3, 900.0)
        t += 3
        assert np.array_equal(np.bincount(occ, minlength=K), counts0)
        assert np.all(st["attempts"] == d.n_sites)
        assert np.all(st["accepted"] <= st["unlike"])
        E += int(st["sum_dE"].sum())
        assert E == orc.energy(d, V, occ)
        assert st["accepted"].sum() > 0


def test_chunking_is_invisible(orc):
    d, V, occ = _setup(orc, 0, (8, 8, 8), 4, 2)
    a, sa = orc.sweeps(d, V, occ, 0, 6, 800.0)
    b, sb1 = orc.sweeps(d, V, occ, 0, 2, 800.0)
    b, sb2 = orc.sweeps(d, V, b, 2, 4, 800.0)
    assert np.array_equal(a, b)
    assert np.array_equal(sa, np.concatenate([sb1, sb2]))


def test_anneal_temperatures(orc):
    """T linear over the call: replaying each sweep alone at its temperature
    gives the same chain."""
    d, V, occ = _setup(orc, 1, (4, 4, 4), 3, 2)
    a, sa = orc.sweeps(d, V, occ, 0, 5, 1500.0, 300.0)
    b = occ
    for i in range(5):
        T = 1500.0 + (300.0 - 1500.0) * i / 4
        b, _ = orc.sweeps(d, V, b, i, 1, T)
    assert np.array_equal(a, b)


def test_beta_zero_accepts_every_unlike(orc):
    d, V, occ = _setup(orc, 0, (6, 6, 6), 4, 3)
    occ2, st = orc.sweeps(d, V, occ, 0, 3, float("inf"))
    assert np.array_equal(st["accepted"], st["unlike"])
    assert st["unlike"].sum() > 0


def test_zero_temperature_never_raises_energy(orc):
    d, V, occ = _setup(orc, 1, (4, 4, 4), 4, 3)
    E = [orc.energy(d, V, occ)]
    t = 0
    for _ in range(6):
        occ, st = orc.sweeps(d, V, occ, t, 1, 0.0)
        t += 1
        E.append(orc.energy(d, V, occ))
    assert all(b <= a for a, b in zip(E, E[1:]))
    assert E[-1] < E[0]


def test_single_species_has_no_unlike(orc):
    d = orc.Desc(0, (4, 4, 4), 1, 2)
    V = inputs.epi_table(2, 1, 0.02, 0)
    occ = np.zeros(d.n_sites, dtype=np.uint8)
    occ2, st = orc.sweeps(d, V, occ, 0, 2, 500.0)
    assert st["unlike"].sum() == 0 and st["accepted"].sum() == 0
    assert np.array_equal(occ, occ2)


@pytest.mark.parametrize("kind,n,K,M", [(0, (12, 12, 12), 4, 3), (1, (8, 8, 8), 5, 4),
                                        (0, (9, 10, 11), 3, 2)])
def test_schedule_independence(orc, kind, n, K, M):
    """Same-colour cells do not interact: visiting them in any order gives the
    same bits."""
    d, V, occ = _setup(orc, kind, n, K, M, seed=3)
    a, sa = orc.sweeps(d, V, occ, 0, 3, 700.0)
    b, sb = orc.sweeps(d, V, occ, 0, 3, 700.0, shuffle_cells=True, shuffle_seed=99)
    assert np.array_equal(a, b)
    assert np.array_equal(sa, sb)


def test_schedule_check_has_teeth(orc):
    """With cells one conventional cell smaller than the rule allows, the
    visiting order of same-colour cells changes the result."""
    d, V, occ = _setup(orc, 0, (12, 12, 12), 4, 3, seed=3)
    L, _ = orc.layout(d)
    a, _ = orc.sweeps(d, V, occ, 0, 2, 700.0, L_override=L - 1)
    b, _ = orc.sweeps(d, V, occ, 0, 2, 700.0, L_override=L - 1, shuffle_cells=True,
                      shuffle_seed=99)
    assert not np.array_equal(a, b)


def test_b2_ground_state(orc):
    """Binary 50/50 BCC with only an attractive unlike first-shell pair
    (V_AB < 0, V_AA = V_BB = 0): the ground state is B2, every site with 8
    unlike nearest neighbours, E = 4 N V_AB, and no configuration lies below
    it.  Slow anneals from several seeds must reach it exactly."""
    n = (4, 4, 4)
    vab = int(round(-0.05 * Q))
    V = np.array([[[0, vab], [vab, 0]]], dtype=np.int64)
    reached = []
    for seed in range(3):
        d = orc.Desc(0, n, 2, 1, seed=seed)
        occ = inputs.initial_occupancy(0, n, 2, seed=seed + 8)
        occ, _ = orc.sweeps(d, V, occ, 0, 3000, 2500.0, 300.0)
        occ, _ = orc.sweeps(d, V, occ, 3000, 20, 0.0)
        E = orc.energy(d, V, occ)
        assert E >= 4 * d.n_sites * vab
        reached.append(E)
        if E == 4 * d.n_sites * vab:
            sub = occ.reshape(-1, 2)
            assert len(set(sub[:, 0])) == 1 and len(set(sub[:, 1])) == 1
            assert sub[0, 0] != sub[0, 1]
    assert min(reached) == 4 * d.n_sites * vab
