"""Pins of the oracle's lattice geometry and link-cell layout (not gpu).

Shell tables are checked against textbook values (tests/golden/shells.json)
and against an independent enumeration of lattice points built from the
conventional cell and its basis; the link-cell edge rule (Sec. 2.2, Eq. 5:
the smallest cell that separates the interactions) is checked from its
geometric criterion.
"""
import itertools

import numpy as np
import pytest

from tests import bruteforce as bf


@pytest.mark.parametrize("kind,name", [(0, "bcc"), (1, "fcc")])
def test_shells_match_textbook(orc, kind, name):
    g = bf.golden("shells.json")[name]
    disp, z, d2 = orc.shells(kind, 4)
    assert list(z) == g["z"]
    assert list(d2) == g["d2"]
    start = 0
    for m in range(4):
        block = disp[start:start + z[m]]
        assert np.all((block ** 2).sum(1) == g["d2"][m])
        assert np.abs(block).max() == g["max_component"][m]
        # sorted lexicographically inside the shell
        assert [tuple(r) for r in block] == sorted(tuple(r) for r in block)
        # closed under inversion
        s = {tuple(r) for r in block}
        assert all(tuple(-np.array(r)) in s for r in s)
        start += z[m]


@pytest.mark.parametrize("kind", [0, 1])
def test_shells_match_independent_enumeration(orc, kind):
    """Lattice points generated as 2*(cell) + basis, classified by length."""
    pts = set()
    for c in itertools.product(range(-3, 4), repeat=3):
        for bv in bf.BASIS[kind]:
            p = tuple(2 * np.array(c) + bv)
            if p != (0, 0, 0):
                pts.add(p)
    lengths = sorted({sum(v * v for v in p) for p in pts})[:4]
    disp, z, d2 = orc.shells(kind, 4)
    start = 0
    for m, L2 in enumerate(lengths):
        want = sorted(p for p in pts if sum(v * v for v in p) == L2)
        got = sorted(tuple(int(v) for v in r) for r in disp[start:start + z[m]])
        assert got == want
        start += z[m]


@pytest.mark.parametrize("kind,M,L_expected", [(0, 1, 2), (0, 2, 2), (0, 3, 2), (0, 4, 3),
                                               (1, 1, 2), (1, 2, 2), (1, 3, 2), (1, 4, 2)])
def test_min_cell_edge(orc, kind, M, L_expected):
    """2L > 1 + h_R: writes of a cell (anchors + partners at <=1 half unit)
    never meet the reads of a same-colour cell (anchors +- (1 + h_R))."""
    disp, z, d2 = orc.shells(kind, M)
    hR = int(np.abs(disp).max())
    L, m = orc.layout(orc.Desc(kind, (24, 24, 24), 2, M))
    assert L == L_expected
    assert 2 * L > 1 + hR and 2 * (L - 1) <= 1 + hR
    assert m == (24 // L - (24 // L) % 2,) * 3


def test_cell_counts_even_or_one(orc):
    for n in range(1, 20):
        L, m = orc.layout(orc.Desc(0, (n, n + 1, n + 2), 2, 2))
        for nd, md in zip((n, n + 1, n + 2), m):
            assert md == 1 or (md % 2 == 0 and md <= nd // L)
            if md == 1:
                assert nd // L < 2
    L, m = orc.layout(orc.Desc(0, (16, 16, 16), 2, 2, flags=orc.FLAG_SINGLE_CELL))
    assert m == (1, 1, 1)


def test_sweep_shift_range_and_spread(orc):
    d = orc.Desc(0, (812, 7, 3), 2, 2, seed=12345)
    shifts = np.array([orc.sweep_shift(d, t) for t in range(2000)])
    for c, nd in enumerate((812, 7, 3)):
        assert shifts[:, c].min() >= 0 and shifts[:, c].max() < nd
    # every residue of the short axes is hit, roughly uniformly
    for c, nd in ((1, 7), (2, 3)):
        h = np.bincount(shifts[:, c], minlength=nd)
        assert h.min() > 2000 / nd * 0.7
    d0 = orc.Desc(0, (8, 8, 8), 2, 2, seed=1, flags=orc.FLAG_NO_SHIFT)
    assert orc.sweep_shift(d0, 5) == (0, 0, 0)
