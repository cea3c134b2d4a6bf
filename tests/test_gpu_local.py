"""The local-energy model on the GPU (the nonlinear short-range model of
Sec. 3): trajectories, statistics and energies equal the oracle's bit for bit
(every kernel trial recomputes the local energies of its interaction zone,
like the oracle's); the linear table reproduces the EPI sweep on the same
link cells; invalid uses are refused."""
import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs
from tests.gpu_util import gpu_lattice, make_case, oracle_desc, require_cuda

pytestmark = pytest.mark.gpu

SCHEDULE = [(2, 1500.0, 800.0), (2, 600.0, 600.0), (1, float("inf"), float("inf")),
            (1, 0.0, 0.0)]


def _table(kind, M, K, seed, scale=0.02):
    from paper_2509_20949_gb300.lattice import local_model_width
    zt = local_model_width(kind, M)
    rng = np.random.default_rng(seed)
    return np.round(rng.normal(0.0, scale, (M, K, K, zt)) * 2.0 ** 32).astype(np.int64)


@pytest.mark.parametrize("kind,n,K,M,pack,scale", [
    (0, (12, 9, 10), 4, 3, 8, 0.02),   # BCC shells 1-3, ragged cells
    (1, (8, 7, 9), 5, 3, 8, 0.02),     # FCC shells 1-3
    (0, (9, 12, 7), 3, 2, 4, 0.02),    # 4-bit storage
    (1, (6, 6, 13), 8, 1, 8, 0.02),    # K = 8, one shell
    (0, (4, 5, 4), 2, 3, 8, 0.02),     # n_d = 4: the smallest lattice, one cell along x and z
    (0, (14, 13, 12), 4, 3, 8, 3.0),   # entries beyond int32: the int64 shared table
])
def test_local_sweeps_match_the_oracle(orc, kind, n, K, M, pack, scale):
    require_cuda()
    case = make_case(kind, n, K, M, seed=31, occ_seed=32)
    T = _table(kind, M, K, seed=33, scale=scale)
    assert (np.abs(T).max() > 2 ** 31) == (scale > 1.0)
    lat = gpu_lattice(case, pack_bits=pack)
    lat.set_local_model(T)
    assert lat.kernel_in_use()[0] == 4
    d = oracle_desc(orc, case)
    assert lat.layout() == orc.local_layout(d)
    occ = case["occ"]
    E0 = orc.local_energy(d, T, occ)
    assert lat.energy() == E0 == lat.running_energy()
    t = 0
    for nsw, a, b in SCHEDULE:
        st = lat.sweep(nsw, a, b)
        occ, per = orc.local_sweeps(d, T, occ, t, nsw, a, b)
        t += nsw
        assert np.array_equal(lat.occupancy(), occ), (nsw, a)
        for key in ("attempts", "unlike", "accepted", "sum_dE"):
            assert st[key] == int(per[key].sum()), key
    assert lat.energy() == orc.local_energy(d, T, occ) == lat.running_energy()


def test_linear_table_is_the_epi_sweep_on_the_same_cells(orc):
    require_cuda()
    from paper_2509_20949_gb300.lattice import local_model_width
    kind, n, K, M = 0, (14, 12, 12), 5, 3
    V = (inputs.epi_table(M, K, 0.03, 5) // 2) * 2
    c = np.arange(local_model_width(kind, M), dtype=np.int64)
    T = (V[:, :, :, None] // 2) * c[None, None, None, :]
    case = make_case(kind, n, K, M, seed=7)
    loc = gpu_lattice(case)
    loc.set_local_model(T)
    L, _ = loc.layout()
    epi_case = dict(case, V=V, min_cell=L)
    epi = gpu_lattice(epi_case)
    assert epi.layout() == loc.layout()
    assert loc.energy() == epi.energy()
    for nsw, a, b in SCHEDULE[:3]:
        assert loc.sweep(nsw, a, b) == epi.sweep(nsw, a, b)
    assert np.array_equal(loc.occupancy(), epi.occupancy())


def test_refusals_and_switching_back(orc):
    require_cuda()
    from paper_2509_20949_gb300 import SmcxError
    from paper_2509_20949_gb300.lattice import local_model_width
    assert local_model_width(0, 4) == 0 and local_model_width(2, 1) == 0
    assert local_model_width(0, 3) == 13 and local_model_width(1, 3) == 25
    big_k = gpu_lattice(make_case(0, (6, 6, 6), 9, 2))
    with pytest.raises(SmcxError):
        big_k.set_local_model(_table(0, 2, 9, 1))
    thin = gpu_lattice(make_case(1, (6, 3, 6), 3, 2))
    with pytest.raises(SmcxError):
        thin.set_local_model(_table(1, 2, 3, 1))
    case = make_case(0, (8, 8, 8), 3, 2, seed=3)
    lat = gpu_lattice(case)
    huge = _table(0, 2, 3, 1)
    huge[0, 0, 0, 0] = 1 << 50
    with pytest.raises(SmcxError):
        lat.set_local_model(huge)
    lat.set_local_model(_table(0, 2, 3, 2))
    with pytest.raises(SmcxError):
        lat.checkpoint()
    lat.sweep(2, 900.0)
    lat.set_epi(case["V"])
    assert lat.kernel_in_use()[0] != 4
    assert lat.energy() == orc.energy(oracle_desc(orc, case), case["V"], lat.occupancy())


@pytest.mark.parametrize("kind,n,K,M", [(0, (22, 20, 24), 5, 3), (1, (16, 15, 17), 4, 3)])
def test_interior_cells_match_the_oracle(orc, kind, n, K, M):
    """Lattices large enough that most cells run the seam-free fast path
    (byte-address deltas), next to the seam cells on the general path."""
    require_cuda()
    case = make_case(kind, n, K, M, seed=41, occ_seed=42)
    T = _table(kind, M, K, seed=43)
    lat = gpu_lattice(case)
    lat.set_local_model(T)
    d = oracle_desc(orc, case)
    occ = case["occ"]
    t = 0
    for nsw, a, b in SCHEDULE[:2]:
        st = lat.sweep(nsw, a, b)
        occ, per = orc.local_sweeps(d, T, occ, t, nsw, a, b)
        t += nsw
        assert np.array_equal(lat.occupancy(), occ)
        assert st["accepted"] == int(per["accepted"].sum()) and st["sum_dE"] == int(per["sum_dE"].sum())
    assert lat.running_energy() == lat.energy() == orc.local_energy(d, T, occ)


def test_colour_phases_over_plane_ranges_equal_the_sweep(orc):
    """Cells of one colour never interact, so running each colour over
    ranges of link-cell z planes (partial windows of the interior-first cell
    order) gives the full sweep's bits."""
    require_cuda()
    case = make_case(0, (26, 18, 30), 4, 3, seed=51, occ_seed=52)
    T = _table(0, 3, 4, seed=53)
    a, b = gpu_lattice(case), gpu_lattice(case)
    a.set_local_model(T)
    b.set_local_model(T)
    _, m = b.layout()
    cuts = [0, 3, 4, m[2] - 2, m[2]]
    for sweep in range(2):
        temp = 900.0
        sa = a.sweep(1, temp)
        tot = dict(attempts=0, unlike=0, accepted=0, sum_dE=0)
        for colour in range(8):
            for lo, hi in zip(cuts, cuts[1:]):
                st = b.run_colour_planes(colour, temp, lo, hi)
                for k in tot:
                    tot[k] += st[k]
        b.sweep_counter = b.sweep_counter + 1
        assert tot == sa
        assert np.array_equal(a.occupancy(), b.occupancy())


def test_bench_local_line(tmp_path):
    require_cuda()
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--mode", "local",
                        "--workload", "bcc16_k4", "--steps", "3", "--warmup", "1",
                        "--no-cpu-baseline"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert line["mode"] == "local" and line["value"] > 0 and line["unit"] == "swaps/s"
    assert line["roofline"]["bound"] == "hbm" and line["gpu_launches"] == 24
