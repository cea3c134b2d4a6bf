"""Directed shell pair counts (Warren-Cowley SRO, Sec. 3.2 Eq. 9) and the
energy from them, through the C ABI, against the oracle's brute-force
counts: row lengths that are and are not multiples of the 128-site spans of
the bit-mask kernel, box rows that do not divide the lattice, 6 species,
BCC shell 4 (two halo rows), FCC shells 1-4, thin lattices, 4-bit storage,
and lattices tall in z whose boxes outnumber the resident blocks, so that a
block walks a run of boxes up a column and carries the halo rows of one
box into the next (ragged last box of a column, runs across columns)."""
import numpy as np
import pytest

from tests.gpu_util import gpu_lattice, make_case, oracle_desc, require_cuda

pytestmark = pytest.mark.gpu

CASES = [
    # kind, n, K, M, pack_bits
    (0, (300, 13, 9), 5, 3, 8),
    (0, (256, 8, 8), 4, 2, 8),
    (0, (129, 17, 10), 6, 4, 8),
    (1, (130, 9, 11), 5, 4, 8),
    (1, (33, 5, 3), 6, 2, 8),
    (0, (31, 3, 2), 3, 3, 8),
    (1, (64, 12, 7), 2, 3, 8),
    (0, (64, 10, 10), 5, 3, 4),
    (1, (130, 9, 11), 5, 4, 4),    # 4-bit storage: FCC, two row groups
    (0, (129, 17, 10), 6, 4, 4),   # 4-bit, K = 6, ragged row length
    (1, (33, 5, 3), 6, 2, 4),
    (0, (31, 3, 2), 3, 3, 4),      # 4-bit, rows shorter than a span (wrap)
    (0, (40, 20, 2602), 5, 3, 8),  # 2 x 651 boxes: carried rows, ragged y and z boxes
    (0, (24, 16, 2800), 4, 4, 8),  # shell 4: two carried halo rows
    (1, (20, 18, 1801), 5, 3, 4),  # FCC, 4-bit storage
]


@pytest.mark.parametrize("kind,n,K,M,pack", CASES)
def test_pair_counts_and_energy_match_oracle(orc, kind, n, K, M, pack):
    require_cuda()
    case = make_case(kind, n, K, M, seed=7, sigma=0.03, epi_seed=8, occ_seed=9)
    lat = gpu_lattice(case, pack_bits=pack)
    d = oracle_desc(orc, case)
    for m in range(1, M + 1):
        cnt, alpha = lat.sro(m)
        assert np.array_equal(cnt, orc.pair_counts(d, case["occ"])[:m]), m
    assert lat.energy() == orc.energy(d, case["V"], case["occ"])
    # after some sweeps (the running energy is checked against the counts)
    lat.sweep(3, 700.0)
    occ = lat.occupancy()
    cnt, _ = lat.sro(M)
    assert np.array_equal(cnt, orc.pair_counts(d, occ))
    assert lat.energy() == lat.running_energy() == orc.energy(d, case["V"], occ)
