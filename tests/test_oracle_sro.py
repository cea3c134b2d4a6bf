"""Pins of the oracle's Warren-Cowley SRO (Sec. 3.2, Eq. 9) (not gpu).

alpha = 0 for a random alloy, < 0 for ordering, > 0 for segregation (the
paper's reading of Eq. 9).  Checked: the sum rule sum_p c_p alpha^{p p'} = 0,
symmetry, the statistical size for a random configuration, and the textbook
perfect-B2 value alpha_1^{AB} = -1.
"""
import math

import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs


@pytest.mark.parametrize("kind,n,K", [(0, (10, 10, 10), 4), (1, (6, 6, 6), 5), (0, (7, 5, 6), 3)])
def test_sum_rule_and_symmetry(orc, kind, n, K):
    d = orc.Desc(kind, n, K, 3)
    occ = inputs.initial_occupancy(kind, n, K, seed=1, fractions=inputs.dirichlet_fractions(K, 5, 1))
    sc = orc.species_counts(occ, K)
    a = orc.sro_alpha(d, orc.pair_counts(d, occ), sc)
    c = sc / sc.sum()
    for m in range(3):
        # sum over neighbour species p of c_p alpha[m][p'][p] = 0 for each centre p'
        assert np.allclose((a[m] * c[None, :]).sum(1), 0.0, atol=1e-12)
        assert np.allclose(a[m], a[m].T, atol=1e-12)


def test_random_configuration_is_near_zero(orc):
    kind, n, K = 0, (16, 16, 16), 4
    d = orc.Desc(kind, n, K, 3)
    occ = inputs.initial_occupancy(kind, n, K, seed=2)
    sc = orc.species_counts(occ, K)
    a = orc.sro_alpha(d, orc.pair_counts(d, occ), sc)
    _, z, _ = orc.shells(kind, 3)
    N = d.n_sites
    c = sc / N
    for m in range(3):
        bound = 5.0 / np.sqrt(N * z[m] * np.outer(c, c))
        assert np.all(np.abs(a[m]) < bound)


def test_perfect_b2(orc):
    n = (6, 6, 6)
    d = orc.Desc(0, n, 2, 2)
    occ = np.tile(np.array([0, 1], dtype=np.uint8), 6 * 6 * 6)
    a = orc.sro_alpha(d, orc.pair_counts(d, occ), orc.species_counts(occ, 2))
    # first shell: all unlike -> P(B|A) = 1, c_B = 1/2 -> alpha = 1 - 2 = -1
    assert a[0, 0, 1] == -1.0 and a[0, 1, 0] == -1.0
    assert a[0, 0, 0] == 1.0
    # second shell: same sublattice -> all like
    assert a[1, 0, 1] == 1.0 and a[1, 0, 0] == -1.0


def test_missing_species_gives_nan(orc):
    d = orc.Desc(0, (4, 4, 4), 3, 1)
    occ = np.tile(np.array([0, 1], dtype=np.uint8), 64)
    a = orc.sro_alpha(d, orc.pair_counts(d, occ), orc.species_counts(occ, 3))
    assert math.isnan(a[0, 2, 0]) and math.isnan(a[0, 0, 2]) and not math.isnan(a[0, 0, 1])
