"""Online kernel choice of a single lattice (SMCX_OPT_KERNEL = 0): the first
colour phases rotate over the kernels that can run the lattice, each timed
three times, and the fastest is kept; results stay bit-identical to the
oracle throughout."""
import numpy as np
import pytest

from tests.gpu_util import gpu_lattice, make_case, oracle_desc, require_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,n,K,M", [(0, (72, 14, 36), 5, 3), (1, (70, 13, 14), 6, 2)])
def test_online_choice_is_bit_exact_and_picks_the_fastest(orc, kind, n, K, M):
    require_cuda()
    case = make_case(kind, n, K, M, seed=41, sigma=0.03, epi_seed=42, occ_seed=43)
    lat = gpu_lattice(case)
    t0 = lat.kernel_tuning()
    assert not t0["done"] and len(t0["candidates"]) >= 2
    kinds = {c["kernel"] for c in t0["candidates"]}
    assert kinds == {2, 3}  # tiled shapes and the cell kernel
    d = oracle_desc(orc, case)
    sweeps, T = 6, 900.0
    o_occ, o_st = orc.sweeps(d, case["V"], case["occ"], 0, sweeps, T)
    for i in range(sweeps):
        s = lat.sweep(1, T)
        o = o_st[i]
        assert (s["attempts"], s["unlike"], s["accepted"], s["sum_dE"]) == \
            (int(o["attempts"]), int(o["unlike"]), int(o["accepted"]), int(o["sum_dE"])), i
    assert np.array_equal(lat.occupancy(), o_occ)
    assert lat.running_energy() == lat.energy() == orc.energy(d, case["V"], o_occ)
    t = lat.kernel_tuning()
    assert t["done"]
    best = min(t["candidates"], key=lambda c: c["best_ms"])
    assert all(c["best_ms"] > 0 for c in t["candidates"])
    kern, shape = lat.kernel_in_use()
    assert (kern, shape) == (best["kernel"], best["shape"])


def test_forced_kernel_is_not_tuned():
    require_cuda()
    case = make_case(0, (72, 14, 36), 4, 2, seed=1)
    lat = gpu_lattice(case, kernel=3)
    assert lat.kernel_tuning()["done"]
    lat.sweep(2, 800.0)
    assert lat.kernel_in_use() == (3, -1)
