"""Bit-exact parity of the cell sweep kernel (one thread per link cell,
global-memory neighbourhoods) and of the generic kernel with the oracle on
small and medium lattices (through the C ABI)."""
import numpy as np
import pytest

from tests.gpu_util import gpu_lattice, make_case, oracle_desc, require_cuda

pytestmark = pytest.mark.gpu

GENERIC, TILED, CELL = 1, 2, 3

CASES = [
    (0, (4, 4, 4), 3, 2),
    (0, (8, 8, 8), 5, 3),
    (1, (8, 8, 8), 4, 3),
    (0, (5, 9, 7), 6, 4),    # ragged edges, K = 6, L = 3
    (1, (9, 6, 11), 2, 4),
    (1, (4, 5, 6), 6, 2),
    (0, (24, 20, 16), 4, 3),
    (1, (20, 18, 22), 5, 3),
]


@pytest.mark.parametrize("kernel", [CELL, GENERIC])
@pytest.mark.parametrize("kind,n,K,M", CASES)
def test_kernel_matches_oracle(orc, kind, n, K, M, kernel):
    require_cuda()
    case = make_case(kind, n, K, M, seed=7, sigma=0.03)
    lat = gpu_lattice(case, kernel=kernel)
    assert lat.kernel_in_use()[0] == kernel
    d = oracle_desc(orc, case)
    o_occ, o_st = orc.sweeps(d, case["V"], case["occ"], 0, 4, 950.0)
    for i in range(4):
        s = lat.sweep(1, 950.0)
        o = o_st[i]
        assert (s["attempts"], s["unlike"], s["accepted"], s["sum_dE"]) == \
            (int(o["attempts"]), int(o["unlike"]), int(o["accepted"]), int(o["sum_dE"])), i
    assert np.array_equal(lat.occupancy(), o_occ)
    assert lat.running_energy() == lat.energy() == orc.energy(d, case["V"], o_occ)


@pytest.mark.parametrize("T", [0.0, float("inf"), 60.0])
def test_cell_temperature_limits(orc, T):
    require_cuda()
    case = make_case(1, (8, 8, 8), 5, 3, seed=2)
    lat = gpu_lattice(case, kernel=CELL)
    d = oracle_desc(orc, case)
    o_occ, _ = orc.sweeps(d, case["V"], case["occ"], 0, 3, T)
    lat.sweep(3, T)
    assert np.array_equal(lat.occupancy(), o_occ)


def test_cell_equals_tiled_on_large_lattice():
    require_cuda()
    case = make_case(0, (68, 12, 36), 5, 3, seed=9, sigma=0.02)
    a = gpu_lattice(case, kernel=CELL)
    b = gpu_lattice(case, kernel=TILED)
    assert a.sweep(5, 1300.0, 500.0) == b.sweep(5, 1300.0, 500.0)
    assert np.array_equal(a.occupancy(), b.occupancy())


def test_unsupported_kernel_request_fails_cleanly():
    require_cuda()
    from paper_2509_20949_gb300 import SmcxError
    case = make_case(0, (3, 3, 3), 3, 2, seed=1)
    lat = gpu_lattice(case, kernel=CELL)
    assert lat.kernel_in_use()[0] == 0
    with pytest.raises(SmcxError):
        lat.sweep(1, 900.0)
