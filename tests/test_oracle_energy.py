"""Pins of the oracle's EPI energy, swap energy change and pair counts (not gpu).

The EPI Hamiltonian is pairwise only (Sec. 3).  The oracle's displacement-list
energy is checked against a brute-force sum over every periodic image of every
site pair (tests/bruteforce.py), including lattices so small that a site is
its own neighbour; the swap energy change computed from the local interaction
zone (Sec. 2.2) is checked against H(after) - H(before).
"""
import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs
from tests import bruteforce as bf

TINY = [
    (0, (1, 1, 1)), (0, (2, 2, 2)), (0, (2, 3, 1)), (0, (3, 3, 3)), (0, (4, 4, 4)),
    (1, (1, 1, 1)), (1, (2, 2, 2)), (1, (1, 2, 3)), (1, (3, 3, 3)),
]


@pytest.mark.parametrize("kind,n", TINY)
@pytest.mark.parametrize("M", [1, 2, 4])
def test_energy_matches_image_brute_force(orc, kind, n, M):
    K = 3
    V = inputs.epi_table(M, K, 0.05, seed=11 * M + kind)
    occ = inputs.initial_occupancy(kind, n, K, seed=3)
    d = orc.Desc(kind, n, K, M)
    assert orc.energy(d, V, occ) == bf.energy(kind, n, V, occ)


@pytest.mark.parametrize("kind,n", TINY)
def test_pair_counts_match_brute_force(orc, kind, n):
    K, M = 3, 4
    occ = inputs.initial_occupancy(kind, n, K, seed=5)
    d = orc.Desc(kind, n, K, M)
    got = orc.pair_counts(d, occ)
    want = bf.pair_counts(kind, n, M, K, occ)
    assert np.array_equal(got.astype(np.int64), want)
    # directed counts are symmetric and sum to N z_m per shell
    assert np.array_equal(got, got.transpose(0, 2, 1))
    _, z, _ = orc.shells(kind, M)
    assert list(got.sum((1, 2))) == [d.n_sites * int(zm) for zm in z]


@pytest.mark.parametrize("kind,n", [(0, (4, 4, 4)), (1, (3, 3, 3)), (0, (2, 2, 2)), (1, (1, 1, 2))])
def test_energy_from_counts_identity(orc, kind, n):
    """H = 1/2 sum_m sum_{p',p} N_m[p'][p] V_m(p', p), exactly."""
    K, M = 4, 3
    V = inputs.epi_table(M, K, 0.03, seed=2)
    occ = inputs.initial_occupancy(kind, n, K, seed=9)
    d = orc.Desc(kind, n, K, M)
    N = orc.pair_counts(d, occ).astype(object)
    tot = sum(int(N[m, a, b]) * int(V[m, a, b]) for m in range(M) for a in range(K) for b in range(K))
    assert tot % 2 == 0
    assert orc.energy(d, V, occ) == tot // 2


@pytest.mark.parametrize("kind,n", [(0, (1, 1, 1)), (0, (2, 2, 2)), (1, (1, 1, 1)), (1, (2, 1, 2)),
                                    (0, (5, 4, 3)), (1, (4, 4, 4))])
def test_delta_e_equals_energy_difference(orc, kind, n):
    K, M = 4, 4
    V = inputs.epi_table(M, K, 0.04, seed=21)
    occ = inputs.initial_occupancy(kind, n, K, seed=4)
    d = orc.Desc(kind, n, K, M)
    N = d.n_sites
    rng = np.random.default_rng(0)
    disp, z, _ = orc.shells(kind, 1)
    E0 = orc.energy(d, V, occ)
    trials = 300 if N > 64 else 150
    for _ in range(trials):
        i, j = (int(v) for v in rng.integers(0, N, 2))
        dE = orc.delta_e(d, V, occ, i, j)
        after = occ.copy()
        after[i], after[j] = occ[j], occ[i]
        assert dE == orc.energy(d, V, after) - E0
