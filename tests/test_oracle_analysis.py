"""Pins of the oracle's analyses (Sec. 3.2): the cylinder composition profile
against a brute-force numpy recount of the definition, the whole-lattice
cylinder against the species counts, and translation covariance."""
import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs

BASIS = {0: [(0, 0, 0), (1, 1, 1)], 1: [(0, 0, 0), (0, 1, 1), (1, 0, 1), (1, 1, 0)]}


def _brute_profile(kind, n, occ, K, axis, o, r2max, length, n_bins):
    nb = len(BASIS[kind])
    out = np.zeros((n_bins, K), dtype=np.uint64)
    idx = 0
    for z in range(n[2]):
        for y in range(n[1]):
            for x in range(n[0]):
                for b in range(nb):
                    h = np.array([2 * x, 2 * y, 2 * z]) + np.array(BASIS[kind][b])
                    rel = [(int(h[d]) - o[d]) % (2 * n[d]) for d in range(3)]
                    t = rel[axis]
                    r2 = 0
                    for d in range(3):
                        if d != axis:
                            v = rel[d] - 2 * n[d] if rel[d] > n[d] else rel[d]
                            r2 += v * v
                    if t < length and r2 <= r2max:
                        out[t * n_bins // length, occ[idx]] += 1
                    idx += 1
    return out


@pytest.mark.parametrize("kind,n,K,axis,o,r2,length,bins", [
    (0, (6, 5, 7), 4, 0, (3, -2, 9), 20, 9, 3),
    (1, (5, 6, 4), 3, 2, (0, 1, 1), 13, 8, 4),
    (0, (4, 4, 9), 2, 2, (1, 1, 17), 8, 18, 6),
])
def test_profile_equals_definition(orc, kind, n, K, axis, o, r2, length, bins):
    occ = inputs.initial_occupancy(kind, n, K, 3, None)
    d = orc.Desc(kind, n, K, 2)
    got = orc.composition_profile(d, occ, axis, o, r2, length, bins)
    assert np.array_equal(got, _brute_profile(kind, n, occ, K, axis, o, r2, length, bins))


def test_whole_lattice_cylinder_counts_every_site(orc):
    kind, n, K = 1, (5, 4, 6), 5
    occ = inputs.initial_occupancy(kind, n, K, 8, None)
    d = orc.Desc(kind, n, K, 2)
    got = orc.composition_profile(d, occ, 1, (0, 0, 0), 10 ** 6, 2 * n[1], 4)
    assert np.array_equal(got.sum(axis=0), np.bincount(occ, minlength=K))
    # 4 bins over 2 n_y = 8 half units: one conventional cell (one y row of 5 x 6 x 4 sites) each
    assert all(int(row.sum()) == n[0] * n[2] * 4 for row in got)


def test_profile_follows_a_translated_lattice(orc):
    """Shifting the cylinder by a conventional cell equals rolling the
    lattice the other way."""
    kind, n, K = 0, (6, 6, 6), 3
    occ = inputs.initial_occupancy(kind, n, K, 4, None)
    d = orc.Desc(kind, n, K, 2)
    a = orc.composition_profile(d, occ, 0, (2, 4, 6), 9, 8, 4)
    grid = occ.reshape(n[2], n[1], n[0], 2)
    rolled = np.roll(grid, shift=(-1, -1, -1), axis=(0, 1, 2)).ravel()  # site (x+1, y+1, z+1) -> (x, y, z)
    b = orc.composition_profile(d, rolled, 0, (0, 2, 4), 9, 8, 4)
    assert np.array_equal(a, b)


def _bfs_clusters(kind, n, occ, species):
    """Breadth-first search over first-shell neighbours, written from the
    geometry (positions 2*(x,y,z) + basis in half units, nearest neighbours
    at squared distance 3 (BCC) or 2 (FCC))."""
    import collections
    import itertools
    nb = len(BASIS[kind])
    d2 = 3 if kind == 0 else 2
    vecs = [v for v in itertools.product(range(-1, 2), repeat=3) if sum(c * c for c in v) == d2] \
        if kind == 0 else [v for v in itertools.product(range(-1, 2), repeat=3)
                           if sum(c * c for c in v) == d2]
    pos_to_site = {}
    sites = []
    for z in range(n[2]):
        for y in range(n[1]):
            for x in range(n[0]):
                for b in range(nb):
                    h = (2 * x + BASIS[kind][b][0], 2 * y + BASIS[kind][b][1], 2 * z + BASIS[kind][b][2])
                    pos_to_site[h] = len(sites)
                    sites.append(h)
    member = np.isin(occ, list(species))
    seen = np.zeros(len(sites), dtype=bool)
    sizes = []
    for s0 in range(len(sites)):
        if not member[s0] or seen[s0]:
            continue
        seen[s0] = True
        q = collections.deque([s0])
        size = 0
        while q:
            s = q.popleft()
            size += 1
            h = sites[s]
            for v in vecs:
                hn = tuple((h[d] + v[d]) % (2 * n[d]) for d in range(3))
                t = pos_to_site[hn]
                if member[t] and not seen[t]:
                    seen[t] = True
                    q.append(t)
        sizes.append(size)
    return sorted(sizes, reverse=True)


@pytest.mark.parametrize("kind,n,K,species", [
    (0, (5, 4, 6), 4, (1,)), (0, (5, 4, 6), 4, (0, 2)), (1, (4, 5, 3), 5, (3,)),
    (1, (4, 5, 3), 5, (0, 1, 4)), (0, (3, 3, 3), 2, (1,))])
def test_clusters_equal_breadth_first_search(orc, kind, n, K, species):
    occ = inputs.initial_occupancy(kind, n, K, 12, None)
    d = orc.Desc(kind, n, K, 2)
    got = [int(v) for v in orc.clusters(d, occ, species)]
    assert got == _bfs_clusters(kind, n, occ, species)
    assert sum(got) == int(np.isin(occ, list(species)).sum())


def test_cluster_limits(orc):
    kind, n, K = 1, (4, 4, 4), 3
    occ = inputs.initial_occupancy(kind, n, K, 2, None)
    d = orc.Desc(kind, n, K, 2)
    assert [int(v) for v in orc.clusters(d, occ, range(K))] == [occ.size]  # periodic lattice: connected
    assert orc.clusters(d, occ, ()).size == 0
