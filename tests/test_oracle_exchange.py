"""Pins of the oracle's replica exchange (Sec. 2.2, Eqs. 6-7) against what
the mathematics fixes: with the replicas' energies frozen, repeated exchange
rounds are a Markov chain on the assignment of replicas to temperatures whose
stationary distribution is the product of the replicas' Boltzmann factors,
prod_k exp(-E_{perm[k]} / (k_B T_k)) (each accepted pair satisfies detailed
balance with respect to it); a sign error in Delta, a wrong beta or a wrong
pair order shifts that distribution.  Also: the even/odd pair schedule and
input checks."""
import itertools

import numpy as np
import pytest

KB = 8.617333262e-5
Q = 2.0 ** -32


def _stationary(E, T):
    perms = list(itertools.permutations(range(len(T))))
    logw = np.array([-sum(E[p[k]] * Q / (KB * T[k]) for k in range(len(T))) for p in perms])
    w = np.exp(logw - logw.max())
    return perms, w / w.sum()


@pytest.mark.parametrize("E_ev,T", [((-0.10, -0.02, 0.05), (300.0, 450.0, 700.0)),
                                    ((0.03, -0.04, 0.0, -0.06), (250.0, 400.0, 600.0, 900.0))])
def test_ladder_samples_the_product_ensemble(orc, E_ev, T):
    E = np.array([int(round(e / Q)) for e in E_ev], dtype=np.int64)
    perms, pi = _stationary(E, T)
    index = {p: i for i, p in enumerate(perms)}
    perm = np.arange(len(T), dtype=np.uint32)
    counts = np.zeros(len(perms))
    rounds = 200_000
    for r in range(rounds):
        perm, _ = orc.exchange(E, T, 1234, r, perm)
        counts[index[tuple(int(v) for v in perm)]] += 1
    freq = counts / rounds
    assert 0.5 * np.abs(freq - pi).sum() < 0.01, (freq, pi)


def test_pair_schedule_and_acceptance_limits(orc):
    T = np.array([100.0, 200.0, 300.0, 400.0, 500.0])
    # energies decreasing along the ladder: every Delta >= 0, always accepted
    E = np.array([5, 4, 3, 2, 1], dtype=np.int64) * (1 << 32)
    p, acc = orc.exchange(E, T, 7, 0, np.arange(5))
    assert list(p) == [1, 0, 3, 2, 4] and list(acc) == [True, False, True, False]
    p, acc = orc.exchange(E, T, 7, 1, np.arange(5))
    assert list(p) == [0, 2, 1, 4, 3] and list(acc) == [False, True, False, True]
    # energies increasing by 100 eV per step: Delta <= -580, exp(Delta) underflows to 0
    E = np.array([1, 2, 3, 4, 5], dtype=np.int64) * (100 << 32)
    for r in range(50):
        p, acc = orc.exchange(E, T, 7, r, np.arange(5))
        assert list(p) == [0, 1, 2, 3, 4] and not acc.any()


def test_rejects_bad_temperatures(orc):
    E = np.zeros(2, dtype=np.int64)
    for T in ([0.0, 300.0], [300.0, float("inf")], [-1.0, 2.0]):
        with pytest.raises(orc.OracleError):
            orc.exchange(E, T, 1, 0, [0, 1])
