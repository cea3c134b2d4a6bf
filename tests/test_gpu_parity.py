"""Bit-exact parity of the CUDA path (through the C ABI) with the oracle.

Every case compares occupancies, per-sweep integer statistics (trials,
unlike trials, accepted swaps, summed energy change), the running and the
recomputed energy and the SRO pair counts element by element: the method's
arithmetic is integer end to end, so the tolerance is zero.
"""
import numpy as np
import pytest

from tests.gpu_util import gpu_lattice, make_case, oracle_desc, require_cuda

pytestmark = pytest.mark.gpu


def _run_both(orc, case, sweeps, T_first, T_last=None, chunks=None, pack_bits=8, kernel=0):
    require_cuda()
    lat = gpu_lattice(case, pack_bits=pack_bits, kernel=kernel)
    d = oracle_desc(orc, case)
    T_last = T_first if T_last is None else T_last
    o_occ, o_st = orc.sweeps(d, case["V"], case["occ"], 0, sweeps, T_first, T_last)
    g_st = []
    if chunks is None:
        for i in range(sweeps):
            T = T_first if sweeps == 1 or T_first == T_last else \
                T_first + (T_last - T_first) * i / (sweeps - 1)
            g_st.append(lat.sweep(1, T))
    else:
        g_tot = lat.sweep(sweeps, T_first, T_last)
        g_st = None
    g_occ = lat.occupancy()
    assert np.array_equal(g_occ, o_occ), "occupancy differs"
    if g_st is not None:
        for i, s in enumerate(g_st):
            o = o_st[i]
            assert (s["attempts"], s["unlike"], s["accepted"], s["sum_dE"]) == \
                (int(o["attempts"]), int(o["unlike"]), int(o["accepted"]), int(o["sum_dE"])), i
    else:
        assert g_tot["accepted"] == int(o_st["accepted"].sum())
        assert g_tot["sum_dE"] == int(o_st["sum_dE"].sum())
    E_o = orc.energy(d, case["V"], o_occ)
    assert lat.energy() == E_o
    assert lat.running_energy() == E_o
    cnt, alpha = lat.sro(case["M"])
    assert np.array_equal(cnt, orc.pair_counts(d, o_occ))
    a_o = orc.sro_alpha(d, cnt, orc.species_counts(o_occ, case["K"]))
    assert np.allclose(alpha, a_o, rtol=1e-13, atol=1e-13, equal_nan=True)
    assert lat.sweep_counter == sweeps
    return lat


def test_philox_device_matches_oracle(orc):
    torch = require_cuda()
    from paper_2509_20949_gb300 import _lib
    L = _lib.lib()
    n = 4096
    out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    key = 0x1234567890ABCDEF
    _lib.check(L.smcx_philox_device(7, 11, 13, 17, key, n, out.data_ptr(), None))
    got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    for i in range(0, n, 97):
        want = orc.philox((7 + i, 11, 13, 17), (key & 0xFFFFFFFF, key >> 32))
        assert list(got[i]) == list(want)


def test_bcc16_k4_full_100_sweeps(orc):
    """BCC 16^3 x2 = 8192 sites, 4 species equiatomic, shells 1-2
    (sigma 0.02 eV, EPI seed 0), 1000 K, 100 sweeps, Philox seed 0."""
    from paper_2509_20949_gb300 import inputs
    w = inputs.workload("bcc16_k4")
    case = make_case(w["kind"], w["n"], w["K"], w["M"], seed=w["seed"], sigma=w["sigma"],
                     epi_seed=w["epi_seed"], occ_seed=w["occ_seed"])
    _run_both(orc, case, w["sweeps"], w["T_first"])


SMALL = [
    # kind, n, K, M, flags, min_cell
    (0, (8, 8, 8), 3, 3, 0, 0),
    (1, (8, 8, 8), 5, 4, 0, 0),
    (0, (9, 7, 11), 4, 2, 0, 0),       # ragged cell edges
    (1, (5, 6, 7), 6, 3, 0, 0),
    (0, (3, 3, 3), 3, 4, 0, 0),        # m = 1 in every dimension
    (1, (2, 2, 2), 2, 2, 0, 0),        # sites that neighbour themselves
    (0, (2, 9, 4), 3, 1, 0, 0),        # mixed m = 1 and m >= 2
    (0, (8, 8, 8), 4, 2, 1, 0),        # no origin shift
    (1, (4, 4, 4), 3, 2, 2, 0),        # single cell
    (0, (12, 12, 12), 4, 3, 0, 3),     # min_cell raises the edge
    (1, (6, 6, 6), 1, 2, 0, 0),        # one species
    (0, (6, 6, 6), 12, 2, 0, 0),       # many species
    (0, (1, 1, 1), 2, 1, 0, 0),        # the smallest lattice: two sites
    (0, (6, 6, 6), 255, 2, 0, 0),      # the largest species count
]


@pytest.mark.parametrize("kind,n,K,M,flags,min_cell", SMALL)
def test_small_lattices(orc, kind, n, K, M, flags, min_cell):
    case = make_case(kind, n, K, M, seed=5, flags=flags, min_cell=min_cell)
    _run_both(orc, case, 6, 900.0)


@pytest.mark.parametrize("pack", [8, 4])
def test_anneal_and_packed_storage(orc, pack):
    case = make_case(0, (10, 10, 10), 5, 3, seed=9, sigma=0.02)
    _run_both(orc, case, 8, 1500.0, 300.0, pack_bits=pack)
    case = make_case(1, (6, 6, 6), 4, 4, seed=3)
    _run_both(orc, case, 5, 1200.0, 600.0, pack_bits=pack, chunks=True)


@pytest.mark.parametrize("T", [0.0, float("inf"), 1.0, 50.0, 1e6])
def test_temperature_limits(orc, T):
    case = make_case(1, (6, 6, 6), 4, 3, seed=2)
    _run_both(orc, case, 3, T)


def test_checkpoint_resume_is_byte_exact(orc):
    require_cuda()
    case = make_case(0, (8, 8, 8), 4, 3, seed=4)
    a = gpu_lattice(case)
    a.sweep(5, 800.0)
    blob = a.checkpoint()
    a.sweep(4, 800.0)
    b = gpu_lattice(case)
    b.restore(blob)
    assert b.sweep_counter == 5
    b.sweep(4, 800.0)
    assert np.array_equal(a.occupancy(), b.occupancy())
    assert a.running_energy() == b.running_energy() == b.energy()
    bad = bytearray(blob)
    bad[100] ^= 1
    with pytest.raises(Exception):
        b.restore(bytes(bad))


def test_occupancy_into_caller_buffer():
    """get_occupancy fills a caller's (pinned) host buffer directly."""
    require_cuda()
    import torch
    case = make_case(0, (12, 10, 8), 4, 2, seed=5)
    lat = gpu_lattice(case)
    lat.sweep(2, 900.0)
    ref = lat.occupancy()
    pinned = torch.empty(lat.N, dtype=torch.uint8, pin_memory=True)
    got = lat.occupancy(out=pinned.numpy())
    assert got.ctypes.data == pinned.data_ptr() and np.array_equal(pinned.numpy(), ref)
    with pytest.raises(ValueError):
        lat.occupancy(out=np.empty(lat.N - 1, dtype=np.uint8))


@pytest.mark.parametrize("kind,n,K,pack", [(0, (13, 7, 9), 5, 8), (1, (5, 11, 6), 6, 8),
                                           (0, (9, 6, 10), 3, 4), (1, (7, 5, 4), 4, 4)])
def test_upload_rejects_bad_ids_and_keeps_the_lattice(orc, kind, n, K, pack):
    """A species id >= K anywhere (head, body or tail of the flat upload)
    raises and leaves the occupancy, and the running energy, as they were; a
    good upload round-trips through the device layout (odd row lengths, both
    storage widths); the running energy's base, taken on first request, equals
    the full energy."""
    require_cuda()
    from paper_2509_20949_gb300 import SmcxError
    case = make_case(kind, n, K, 3, seed=12)
    lat = gpu_lattice(case, pack_bits=pack)
    lat.sweep(3, 800.0)
    before = lat.occupancy()
    e_run = lat.running_energy()
    assert e_run == lat.energy() == orc.energy(oracle_desc(orc, case), case["V"], before)
    for pos in (0, 7, lat.N // 2 + 3, lat.N - 1):
        bad = before.copy()
        bad[pos] = K
        with pytest.raises(SmcxError):
            lat.set_occupancy(bad)
        assert np.array_equal(lat.occupancy(), before)
        assert lat.running_energy() == e_run
    other = make_case(kind, n, K, 3, occ_seed=99)["occ"]
    lat.set_occupancy(other)
    assert np.array_equal(lat.occupancy(), other)
    lat.sweep(2, 600.0)
    assert lat.running_energy() == lat.energy()
