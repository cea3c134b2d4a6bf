"""The oracle's OpenMP variants (not gpu): the cells of one colour shared
out over threads give the sequential oracle's occupancy and per-sweep
statistics bit for bit (cells of one colour never interact, Sec. 2.2), for
any thread count.  They serve the CPU baseline on all host cores and the
whole-phase replays of the 1.07e9-site lattice."""
import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs


@pytest.mark.parametrize("kind,n,K,M,T0,T1", [
    (0, (16, 16, 16), 4, 2, 1000.0, 1000.0),
    (0, (21, 18, 23), 5, 3, 1200.0, 600.0),      # ragged link cells, anneal
    (1, (12, 13, 12), 5, 4, 800.0, 800.0),
    (1, (10, 10, 10), 3, 3, float("inf"), float("inf")),
    (0, (12, 12, 12), 3, 2, 0.0, 0.0),
])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_sweeps_par_equals_sequential(orc, kind, n, K, M, T0, T1, threads):
    V = inputs.epi_table(M, K, 0.03, 5)
    occ = inputs.initial_occupancy(kind, n, K, 6)
    d = orc.Desc(kind, n, K, M, seed=77)
    a, sa = orc.sweeps(d, V, occ, 4, 3, T0, T1)
    b, sb = orc.sweeps_par(d, V, occ, 4, 3, T0, T1, n_threads=threads)
    assert np.array_equal(a, b)
    assert np.array_equal(sa, sb)


@pytest.mark.parametrize("threads", [2, 8])
def test_phase_cells_par_equals_sequential(orc, threads):
    V = inputs.epi_table(3, 5, 0.02, 1)
    occ = inputs.initial_occupancy(0, (30, 28, 26), 5, 2)
    d = orc.Desc(0, (30, 28, 26), 5, 3, seed=3)
    L, m = orc.layout(d)
    for colour in (0, 5):
        bits = [(colour >> a) & 1 for a in range(3)]
        cids = np.array([cid for cid in range(m[0] * m[1] * m[2])
                         if (cid % m[0]) % 2 == bits[0] and ((cid // m[0]) % m[1]) % 2 == bits[1]
                         and (cid // (m[0] * m[1])) % 2 == bits[2]], dtype=np.uint32)
        a, sa = orc.phase_cells(d, V, occ, 9, 700.0, colour, cids)
        b, sb = orc.phase_cells_par(d, V, occ, 9, 700.0, colour, cids, n_threads=threads)
        assert np.array_equal(a, b)
        assert sa == sb
        # a cell of another colour is rejected, as by the sequential replay
        with pytest.raises(orc.OracleError):
            orc.phase_cells_par(d, V, occ, 9, 700.0, colour ^ 1, cids[:1], n_threads=threads)
