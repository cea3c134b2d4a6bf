"""Pins of the oracle's random-number keying and schedule (not gpu).

The paper fixes none of these; the project's specification does (the
readings of the RNG, the per-sweep origin shift and the trial order).  Here
they are re-derived by hand, trial by trial, from primitives that are pinned
elsewhere -- Philox4x32-10 (its published known-answer vectors, below), the
energy change of one swap (H(after) - H(before), test_oracle_energy.py) and
the threshold tables (the closed form exp(-beta dE), Sec. 2.1 Eq. 3) -- and
compared with what the oracle's sweep does:

  * origin shift of sweep t: w = Philox(counter (0, 0, t, 1), key seed),
    s_d = floor(w_d n_d / 2^32) for d = x, y, z (the "dynamically
    constructed" link cells of Sec. 2.2);
  * trial k of link cell cid in sweep t: w = Philox(counter (k >> 1, cid, t,
    0), key (seed_lo, seed_hi)); words 2(k & 1) and 2(k & 1) + 1 are the
    partner choice and the Metropolis variate; the partner is first-shell
    direction floor(w_a z_1 / 2^32) of the lexicographically sorted shell;
  * sites of a cell in raster order: basis fastest, then shifted x, y, z.
A wrong word, counter slot, key half, dimension or visiting order in the
oracle fails these checks.
"""
import itertools

import numpy as np
import pytest

from tests import bruteforce as bf

MASK32 = (1 << 32) - 1


def test_philox_known_answer_vectors(orc):
    """Philox4x32-10 against the Random123 known-answer vectors."""
    for v in bf.golden("philox_kat.json")["philox4x32_10"]:
        c = [int(x, 16) for x in v["counter"]]
        k = [int(x, 16) for x in v["key"]]
        want = [int(x, 16) for x in v["out"]]
        assert [int(x) for x in orc.philox(c, k)] == want


def _key(seed):
    return (seed & MASK32, seed >> 32)


@pytest.mark.parametrize("n,seed", [((812, 7, 3), 12345), ((30, 31, 32), (7 << 32) | 99),
                                    ((5, 64, 1000), 2 ** 63 + 17)])
def test_sweep_shift_by_hand(orc, n, seed):
    d = orc.Desc(0, n, 2, 2, seed=seed)
    for t in (0, 1, 2, 777, 2 ** 31 + 5):
        w = orc.philox((0, 0, t, 1), _key(seed))
        want = tuple(int((int(w[c]) * n[c]) >> 32) for c in range(3))
        assert orc.sweep_shift(d, t) == want


def _first_shell(kind):
    """Lexicographically sorted first-shell vectors in half units (textbook)."""
    if kind == 0:
        vecs = list(itertools.product((-1, 1), repeat=3))
    else:
        vecs = [v for v in itertools.product((-1, 0, 1), repeat=3)
                if sorted(abs(c) for c in v) == [0, 1, 1]]
    return sorted(vecs)


def _site(kind, n, h):
    """Canonical index of the site at half-unit position h (periodic)."""
    h = [h[c] % (2 * n[c]) for c in range(3)]
    cell = [h[c] // 2 for c in range(3)]
    par = tuple(h[c] & 1 for c in range(3))
    b = [tuple(v) for v in bf.BASIS[kind]].index(par)
    return ((cell[2] * n[1] + cell[1]) * n[0] + cell[0]) * len(bf.BASIS[kind]) + b


def _accept(dE, wb, T, orc):
    tab, s, mode = orc.thresholds(T)
    if dE <= 0 or mode == orc.MODE_ACCEPT_ALL:
        return True
    if mode == orc.MODE_ZERO_T:
        return False
    idx = dE >> s
    if idx >= 1 << 27:
        return False
    thr = (((int(tab[0, idx & 511]) * int(tab[1, (idx >> 9) & 511])) >> 32)
           * int(tab[2, idx >> 18])) >> 32
    return wb < thr


def _replay_cell_by_hand(orc, d, V, occ, t, T, cid):
    """The trials of link cell cid of sweep t, from the specification."""
    kind, n = d.kind, d.n
    nb = len(bf.BASIS[kind])
    L, m = orc.layout(d)
    c = (cid % m[0], (cid // m[0]) % m[1], cid // (m[0] * m[1]))
    lo = [c[a] * n[a] // m[a] for a in range(3)]
    hi = [(c[a] + 1) * n[a] // m[a] for a in range(3)]
    w = orc.philox((0, 0, t, 1), _key(d.seed))
    shift = [int((int(w[a]) * n[a]) >> 32) for a in range(3)]
    s1 = _first_shell(kind)
    occ = occ.copy()
    st = dict(attempts=0, unlike=0, accepted=0, sum_dE=0)
    k = 0
    for zs in range(lo[2], hi[2]):
        for ys in range(lo[1], hi[1]):
            for xs in range(lo[0], hi[0]):
                for b in range(nb):
                    x, y, z = ((xs + shift[0]) % n[0], (ys + shift[1]) % n[1],
                               (zs + shift[2]) % n[2])
                    hpos = [2 * x + bf.BASIS[kind][b][0], 2 * y + bf.BASIS[kind][b][1],
                            2 * z + bf.BASIS[kind][b][2]]
                    i = _site(kind, n, hpos)
                    ww = orc.philox((k >> 1, cid, t, 0), _key(d.seed))
                    wa, wb = int(ww[2 * (k & 1)]), int(ww[2 * (k & 1) + 1])
                    dvec = s1[(wa * len(s1)) >> 32]
                    j = _site(kind, n, [hpos[a] + dvec[a] for a in range(3)])
                    st["attempts"] += 1
                    k += 1
                    if occ[i] == occ[j]:
                        continue
                    st["unlike"] += 1
                    dE = orc.delta_e(d, V, occ, i, j)
                    if _accept(dE, wb, T, orc):
                        occ[i], occ[j] = occ[j], occ[i]
                        st["accepted"] += 1
                        st["sum_dE"] += dE
    return occ, st


@pytest.mark.parametrize("kind,n,K,M,T,t", [
    (0, (8, 8, 8), 3, 2, 900.0, 5),
    (0, (9, 10, 11), 4, 3, 400.0, 2 ** 31 + 3),   # ragged cells, large sweep index
    (1, (8, 9, 8), 3, 2, 1500.0, 11),
    (1, (6, 6, 7), 5, 4, float("inf"), 1),
    (0, (8, 8, 9), 2, 1, 0.0, 4),
])
def test_cell_trials_by_hand(orc, kind, n, K, M, T, t):
    """Every trial of several link cells (each colour) re-derived from the
    keying and the schedule matches the oracle's replay, occupancy and
    integer statistics."""
    from paper_2509_20949_gb300 import inputs
    seed = (0x5EED << 32) | 0xC0FFEE
    V = inputs.epi_table(M, K, 0.05, 3)
    occ = inputs.initial_occupancy(kind, n, K, 21)
    d = orc.Desc(kind, n, K, M, seed=seed)
    L, m = orc.layout(d)
    rng = np.random.default_rng(4)
    checked = 0
    for colour in range(8):
        bits = [(colour >> a) & 1 for a in range(3)]
        cells = [cid for cid in range(m[0] * m[1] * m[2])
                 if all(((cid // [1, m[0], m[0] * m[1]][a]) % m[a]) % 2 == bits[a]
                        for a in range(3))]
        if not cells:
            continue
        cid = int(rng.choice(cells))
        want_occ, want = _replay_cell_by_hand(orc, d, V, occ, t, T, cid)
        got_occ, got = orc.phase_cells(d, V, occ, t, T, colour, np.array([cid], dtype=np.uint32))
        assert np.array_equal(got_occ, want_occ), (colour, cid)
        assert {k: int(v) for k, v in got.items()} == want, (colour, cid)
        checked += 1
    assert checked == 8
