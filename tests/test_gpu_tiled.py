"""Bit-exact parity of the tiled shared-memory sweep kernel (through the C
ABI) with the oracle and with the generic kernel, from lattices that span
several tiles with ragged cell edges and seam-crossing tiles up to the
1.07e9-site lattice of the benchmark (sampled link cells there)."""
import numpy as np
import pytest

from tests.gpu_util import (colour_cells, gpu_lattice, make_case, oracle_desc, require_cuda,
                            write_region_sites)

pytestmark = pytest.mark.gpu

GENERIC, TILED = 1, 2


def _compare_sweeps(orc, case, sweeps, T, pack_bits=8, shape=None, staging=None):
    require_cuda()
    lat = gpu_lattice(case, pack_bits=pack_bits, kernel=TILED)
    if shape is not None:
        lat.set_option(2, shape)
    if staging is not None:
        lat.set_option(3, staging)
    kern, sh = lat.kernel_in_use()
    assert kern == TILED
    d = oracle_desc(orc, case)
    o_occ, o_st = orc.sweeps(d, case["V"], case["occ"], 0, sweeps, T)
    for i in range(sweeps):
        s = lat.sweep(1, T)
        o = o_st[i]
        assert (s["attempts"], s["unlike"], s["accepted"], s["sum_dE"]) == \
            (int(o["attempts"]), int(o["unlike"]), int(o["accepted"]), int(o["sum_dE"])), i
    assert np.array_equal(lat.occupancy(), o_occ)
    E = orc.energy(d, case["V"], o_occ)
    assert lat.running_energy() == E == lat.energy()
    return lat


CASES = [
    # kind, n, K, M
    (0, (68, 12, 20), 4, 2),
    (0, (71, 13, 21), 5, 3),       # ragged edges in every dimension
    (0, (70, 12, 22), 6, 3),       # K = 6 (5-bit fields)
    (0, (104, 18, 30), 3, 4),      # shells 1-4: L = 3
    (1, (68, 12, 12), 5, 4),
    (1, (69, 13, 14), 4, 3),
    (1, (70, 12, 13), 6, 2),
    (0, (68, 12, 20), 2, 3),
]


@pytest.mark.parametrize("kind,n,K,M", CASES)
def test_tiled_matches_oracle(orc, kind, n, K, M):
    case = make_case(kind, n, K, M, seed=11, sigma=0.03)
    _compare_sweeps(orc, case, 3, 850.0)


@pytest.mark.parametrize("pack", [8, 4])
@pytest.mark.parametrize("shape", [0, 1])
def test_tiled_shapes_and_packing(orc, pack, shape):
    case = make_case(0, (69, 12, 36), 5, 3, seed=2, sigma=0.02)
    _compare_sweeps(orc, case, 2, 1100.0, pack_bits=pack, shape=shape)
    case = make_case(0, (68, 12, 36), 6, 2, seed=4, sigma=0.02)  # uniform edges
    _compare_sweeps(orc, case, 2, 900.0, pack_bits=pack, shape=shape)
    case = make_case(1, (68, 13, 20), 4, 4, seed=5, sigma=0.02)
    _compare_sweeps(orc, case, 2, 700.0, pack_bits=pack, shape=shape)


@pytest.mark.parametrize("pack", [8, 4])
@pytest.mark.parametrize("staging", [0, 1])
def test_tiled_staging_paths(orc, pack, staging):
    """Tiles filled by bulk (TMA) copies of each row's 16-byte aligned span
    (staging 0, wherever it fits; 8-byte cp.async copies elsewhere) and by
    8-byte copies only (staging 1): eight sweeps each, so the per-sweep origin
    shifts put the tile rows at many alignments, including tiles across the
    periodic seams; uniform and ragged x edges."""
    case = make_case(0, (68, 12, 36), 5, 3, seed=31, sigma=0.02)    # uniform edges
    _compare_sweeps(orc, case, 8, 1000.0, pack_bits=pack, staging=staging)
    case = make_case(1, (68, 13, 21), 4, 3, seed=32, sigma=0.02)    # FCC, ragged y and z
    _compare_sweeps(orc, case, 8, 900.0, pack_bits=pack, staging=staging)
    case = make_case(0, (71, 12, 20), 5, 2, seed=33, sigma=0.03)    # ragged x: copies only
    _compare_sweeps(orc, case, 4, 1300.0, pack_bits=pack, staging=staging)


@pytest.mark.parametrize("pack", [8, 4])
def test_tiled_wide_warp_shape(orc, pack):
    """Tile shape 2: warps of 32 link cells along x (a tile needs one more
    active cell than it holds along each axis: BCC 32 x 1 x 8, FCC 32 x 1 x
    4): uniform and ragged edges, BCC and FCC, both storages."""
    case = make_case(0, (136, 8, 36), 5, 3, seed=21, sigma=0.02)    # uniform edges
    _compare_sweeps(orc, case, 2, 1150.0, pack_bits=pack, shape=2)
    case = make_case(0, (139, 11, 39), 4, 2, seed=22, sigma=0.03)   # ragged in every dimension
    _compare_sweeps(orc, case, 2, 800.0, pack_bits=pack, shape=2)
    case = make_case(1, (137, 9, 21), 5, 3, seed=23, sigma=0.02)    # FCC, ragged
    _compare_sweeps(orc, case, 2, 1000.0, pack_bits=pack, shape=2)
    case = make_case(0, (136, 10, 38), 6, 3, seed=24, sigma=0.02)   # K = 6
    _compare_sweeps(orc, case, 2, 600.0, pack_bits=pack, shape=2)


@pytest.mark.parametrize("T", [0.0, float("inf"), 100.0])
def test_tiled_temperature_limits(orc, T):
    case = make_case(0, (68, 12, 20), 4, 3, seed=8)
    _compare_sweeps(orc, case, 2, T)


def test_tiled_equals_generic_anneal():
    require_cuda()
    case = make_case(1, (70, 14, 14), 5, 3, seed=3, sigma=0.02)
    a = gpu_lattice(case, kernel=TILED)
    b = gpu_lattice(case, kernel=GENERIC)
    sa = a.sweep(6, 1500.0, 400.0)
    sb = b.sweep(6, 1500.0, 400.0)
    assert sa == sb
    assert np.array_equal(a.occupancy(), b.occupancy())


def test_fcc128_k5_full_size_colour_phases(orc):
    """FCC 128^3 x4 = 8.4M sites, Dirichlet(5) composition, shells 1-4 at
    800 K (the oracle replays two complete colour phases)."""
    require_cuda()
    from paper_2509_20949_gb300 import inputs
    w = inputs.workload("fcc128_k5")
    case = make_case(w["kind"], w["n"], w["K"], w["M"], seed=w["seed"], sigma=w["sigma"],
                     epi_seed=w["epi_seed"], occ_seed=w["occ_seed"], fractions=w["fractions"])
    lat = gpu_lattice(case, kernel=TILED)
    assert lat.kernel_in_use()[0] == TILED
    d = oracle_desc(orc, case)
    lat.sweep(1, w["T_first"])  # sweep 0 on the GPU, then replay phases of sweep 1
    occ = lat.occupancy()
    for colour in (0, 5):
        g = lat.run_colour(colour, w["T_first"])
        o_occ, o = orc.phase_cells(d, case["V"], occ, 1, w["T_first"], colour,
                                   colour_cells(orc, d, colour))
        occ = lat.occupancy()
        assert np.array_equal(occ, o_occ)
        assert (g["attempts"], g["unlike"], g["accepted"], g["sum_dE"]) == \
            (o["attempts"], o["unlike"], o["accepted"], o["sum_dE"])


def test_bcc812_k5_sampled_cells_and_invariants(orc):
    """BCC 812^3 x2 = 1.07e9 sites (the benchmark lattice, tiled kernel):
    the trials of 3000 sampled link cells of two colour phases match the
    oracle bit for bit; species counts are conserved and the running energy
    equals the recomputed energy after a full sweep."""
    require_cuda()
    from paper_2509_20949_gb300 import inputs
    w = inputs.workload("bcc812_k5")
    case = make_case(w["kind"], w["n"], w["K"], w["M"], seed=w["seed"], sigma=w["sigma"],
                     epi_seed=w["epi_seed"], occ_seed=w["occ_seed"])
    lat = gpu_lattice(case, kernel=TILED)
    assert lat.kernel_in_use()[0] == TILED
    d = oracle_desc(orc, case)
    counts0 = np.bincount(case["occ"], minlength=w["K"])
    rng = np.random.default_rng(5)
    T = 1200.0
    before = case["occ"]
    for colour in (0, 6):
        g = lat.run_colour(colour, T)
        after = lat.occupancy()
        cids = colour_cells(orc, d, colour)
        pick = np.sort(rng.choice(cids, 3000, replace=False)).astype(np.uint32)
        o_occ, _ = orc.phase_cells(d, case["V"], before, 0, T, colour, pick)
        sites = write_region_sites(orc, d, 0, pick)
        assert np.array_equal(after[sites], o_occ[sites])
        assert g["attempts"] == len(cids) * 16
        before = after
    lat.sweep_counter = 0
    lat.sweep(1, T)
    final = lat.occupancy()
    assert np.array_equal(np.bincount(final, minlength=w["K"]), counts0)
    assert lat.running_energy() == lat.energy()
