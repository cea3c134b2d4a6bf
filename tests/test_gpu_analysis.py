"""Analyses of Sec. 3.2 through the C ABI, against the oracle: composition
profiles along cylinders (the paper's atom-probe cylinders r = 12a, l = 72a
included), cluster (precipitate) sizes, configuration-averaged SRO."""
import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs
from tests.gpu_util import gpu_lattice, make_case, oracle_desc, require_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,n,K,pack,axis,o,r2,length,bins", [
    (0, (20, 18, 22), 5, 8, 2, (7, -3, 40), 50, 30, 6),
    (1, (16, 14, 12), 4, 8, 0, (3, 3, 3), 20, 32, 8),
    (0, (12, 12, 12), 6, 4, 1, (0, 0, 0), 10 ** 6, 24, 12),
    (0, (13, 10, 9), 9, 8, 0, (30, 5, -7), 40, 20, 5),   # n_x % 4 != 0, K > 6 (codes = ids)
    (1, (7, 9, 11), 6, 8, 2, (1, 2, 3), 12, 22, 11),     # K = 6 (codes 5 sigma), short rows
    (1, (9, 8, 10), 5, 4, 1, (4, 40, 2), 30, 16, 4),     # FCC, 4-bit storage, axis y
    (0, (12, 10, 9), 12, 8, 2, (3, 4, 5), 60, 18, 6),    # K > 8 along z: warp-combined atomics
])
def test_profile_matches_oracle(orc, kind, n, K, pack, axis, o, r2, length, bins):
    require_cuda()
    case = make_case(kind, n, K, 2, seed=3)
    lat = gpu_lattice(case, pack_bits=pack)
    lat.sweep(2, 900.0)
    occ = lat.occupancy()
    d = oracle_desc(orc, case)
    got = lat.composition_profile(axis, o, r2, length, bins)
    assert np.array_equal(got, orc.composition_profile(d, occ, axis, o, r2, length, bins))


def test_paper_apt_cylinder(orc):
    """r = 12a (24 half units), l = 72a (144 half units) along z through the
    middle of a BCC 80^3 lattice, 18 bins of 4a."""
    require_cuda()
    case = make_case(0, (80, 80, 80), 5, 3, seed=5, sigma=0.02)
    lat = gpu_lattice(case)
    lat.sweep(3, 800.0)
    occ = lat.occupancy()
    d = oracle_desc(orc, case)
    got = lat.composition_profile(2, (80, 80, 8), 24 * 24, 144, 18)
    assert np.array_equal(got, orc.composition_profile(d, occ, 2, (80, 80, 8), 576, 144, 18))
    assert got.sum() > 0


@pytest.mark.parametrize("kind,n,K,pack,species", [
    (0, (24, 20, 16), 5, 8, (4,)), (0, (24, 20, 16), 5, 8, (0, 1)),
    (1, (14, 12, 10), 4, 8, (2,)), (1, (14, 12, 10), 4, 4, (0, 1, 3)),
    (0, (10, 10, 10), 3, 8, (0, 1, 2)),     # every site: one cluster
])
def test_clusters_match_oracle(orc, kind, n, K, pack, species):
    require_cuda()
    case = make_case(kind, n, K, 2, seed=6)
    lat = gpu_lattice(case, pack_bits=pack)
    lat.sweep(2, 600.0)
    occ = lat.occupancy()
    d = oracle_desc(orc, case)
    want = orc.clusters(d, occ, species)
    got = lat.clusters(species)
    assert np.array_equal(got, want)
    assert np.array_equal(lat.clusters(species, cap=3), want[:3])


def test_sro_average_is_the_mean_over_snapshots():
    require_cuda()
    case = make_case(0, (12, 12, 12), 4, 3, seed=8)
    a = gpu_lattice(case)
    b = gpu_lattice(case)
    tot, mean_alpha = a.sro_average(3, 4, 5, 700.0)
    counts, alphas = None, []
    for _ in range(4):
        b.sweep(5, 700.0)
        c, al = b.sro(3)
        counts = c if counts is None else counts + c
        alphas.append(al)
    assert np.array_equal(tot, counts)
    assert np.allclose(mean_alpha, np.mean(alphas, axis=0), rtol=0, atol=0)
