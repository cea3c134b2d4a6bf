"""Long-run parity (the segment checks of long runs): the GPU runs a lattice
through a 10^4-sweep linear anneal (1200 -> 600 K, the schedule of the
1.07e9-site workload) with checkpoints, and from the checkpoints at sweeps
0, 5000 and 9997 the oracle replays 3 sweeps that must end in the GPU's
bits; the FCC 128^3 workload runs its 1000 sweeps with oracle checks every
100 sweeps and segment replays.  On the 1.07e9-site lattice itself sampled
link cells of colour phases after 200 GPU sweeps are replayed (whole phases
are in test_gpu_fullsize.py)."""
import numpy as np
import pytest

from tests.gpu_util import (colour_cells, gpu_lattice, make_case, oracle_desc, require_cuda,
                            write_region_sites)

pytestmark = pytest.mark.gpu

N_SWEEPS, T0, T1 = 10000, 1200.0, 600.0


def anneal_T(t):
    return T0 + (T1 - T0) * t / (N_SWEEPS - 1)


def test_anneal_segments_match_oracle(orc):
    require_cuda()
    case = make_case(0, (96, 96, 96), 5, 3, seed=11, sigma=0.02, epi_seed=12, occ_seed=13)
    lat = gpu_lattice(case)
    d = oracle_desc(orc, case)
    # GPU segments [0, 5000), [5000, 9997), [9997, 10000); each call interpolates
    # its own first and last temperature of the global schedule
    bounds = [0, 5000, 9997, N_SWEEPS]
    ckpt = {}
    for a, b in zip(bounds[:-1], bounds[1:]):
        ckpt[a] = lat.checkpoint()
        assert lat.sweep_counter == a
        lat.sweep(b - a, anneal_T(a), anneal_T(b - 1))
    final = lat.occupancy()
    E_final = lat.running_energy()
    assert E_final == lat.energy()
    for a in (0, 5000, 9997):
        lat.restore(ckpt[a])
        start = lat.occupancy()
        g = lat.sweep(3, anneal_T(a), anneal_T(a + 2))
        o_occ, o_st = orc.sweeps(d, case["V"], start, a, 3, anneal_T(a), anneal_T(a + 2))
        assert np.array_equal(lat.occupancy(), o_occ), a
        assert g["accepted"] == int(o_st["accepted"].sum()) and g["sum_dE"] == int(o_st["sum_dE"].sum())
        if a == 9997:
            assert np.array_equal(o_occ, final)
            assert lat.running_energy() == E_final


def test_bcc812_sampled_cells_after_200_sweeps(orc):
    """The 1.07e9-site lattice after 200 annealing sweeps on the GPU: 2000
    sampled link cells of two colour phases of sweep 200 match the oracle."""
    require_cuda()
    from paper_2509_20949_gb300 import inputs
    w = inputs.workload("bcc812_k5")
    case = make_case(w["kind"], w["n"], w["K"], w["M"], seed=w["seed"], sigma=w["sigma"],
                     epi_seed=w["epi_seed"], occ_seed=w["occ_seed"])
    lat = gpu_lattice(case)
    d = oracle_desc(orc, case)
    lat.sweep(200, anneal_T(0), anneal_T(199))
    assert lat.sweep_counter == 200
    before = lat.occupancy()
    rng = np.random.default_rng(17)
    T = anneal_T(200)
    for colour in (3, 4):
        lat.run_colour(colour, T)
        after = lat.occupancy()
        pick = np.sort(rng.choice(colour_cells(orc, d, colour), 2000, replace=False)).astype(np.uint32)
        o_occ, _ = orc.phase_cells(d, case["V"], before, 200, T, colour, pick)
        sites = write_region_sites(orc, d, 200, pick)
        assert np.array_equal(after[sites], o_occ[sites]), colour
        before = after
    assert lat.running_energy() == lat.energy()


def test_fcc128_k5_thousand_sweeps_with_sro_checks(orc):
    """FCC 128^3 x4 = 8.4e6 sites, K = 5 (Dirichlet(5) composition), shells
    1-4, 800 K, 1000 sweeps on the GPU.  Every 100 sweeps the SRO pair counts
    equal the oracle's counts of the GPU's occupancy (and satisfy the sum
    rule), the full energy equals the oracle's and the running energy (its
    base taken at set_epi), and the species counts are conserved.  From the
    GPU's states at sweeps 0, 500 and 997 the oracle replays 3 sweeps (cells
    of each colour over all host cores) that end in the GPU's bits with the
    same per-sweep statistics."""
    require_cuda()
    from paper_2509_20949_gb300 import inputs
    w = inputs.workload("fcc128_k5")
    case = make_case(w["kind"], w["n"], w["K"], w["M"], seed=w["seed"], sigma=w["sigma"],
                     epi_seed=w["epi_seed"], occ_seed=w["occ_seed"], fractions=w["fractions"])
    lat = gpu_lattice(case)
    d = oracle_desc(orc, case)
    T = w["T_first"]
    counts0 = np.bincount(case["occ"], minlength=w["K"])
    c = counts0 / counts0.sum()
    seg_starts = (0, 500, 997)
    marks = sorted((set(range(100, 1001, 100)) | set(seg_starts) | {a + 3 for a in seg_starts})
                   - {0})
    states, seg_stats, t = {0: case["occ"]}, {}, 0
    for mark in marks:
        st = lat.sweep(mark - t, T)
        if t in seg_starts:
            assert mark == t + 3
            seg_stats[t] = st
        t = mark
        if t in seg_starts or t - 3 in seg_starts:
            states[t] = lat.occupancy()
        if t % 100 == 0:
            occ = lat.occupancy()
            assert np.array_equal(np.bincount(occ, minlength=w["K"]), counts0)
            cnt, alpha = lat.sro(w["M"])
            assert np.array_equal(cnt, orc.pair_counts(d, occ)), t
            E = lat.energy()
            assert E == orc.energy(d, case["V"], occ) == lat.running_energy(), t
            for m in range(w["M"]):
                assert np.allclose(alpha[m] @ c, 0.0, atol=1e-12)  # sum_p c_p alpha^{pp'} = 0
    assert lat.sweep_counter == 1000
    for a in seg_starts:
        o_occ, o_st = orc.sweeps_par(d, case["V"], states[a], a, 3, T)
        assert np.array_equal(o_occ, states[a + 3]), a
        g = seg_stats[a]
        assert (g["attempts"], g["unlike"], g["accepted"], g["sum_dE"]) == tuple(
            int(o_st[k].sum()) for k in ("attempts", "unlike", "accepted", "sum_dE")), a


def test_bcc812_packed_storage_equals_bytes():
    """The 1.07e9-site lattice in 4-bit packed storage (0.54 GB) runs the same
    trajectory as in 8-bit storage."""
    require_cuda()
    import torch
    from paper_2509_20949_gb300 import inputs
    w = inputs.workload("bcc812_k5")
    case = make_case(w["kind"], w["n"], w["K"], w["M"], seed=w["seed"], sigma=w["sigma"],
                     epi_seed=w["epi_seed"], occ_seed=w["occ_seed"])
    res = []
    for pack in (8, 4):
        lat = gpu_lattice(case, pack_bits=pack)
        st = lat.sweep(2, anneal_T(0), anneal_T(1))
        res.append((lat.occupancy(), st, lat.running_energy()))
        lat.close()
        del lat
        torch.cuda.empty_cache()
    assert res[0][1] == res[1][1] and res[0][2] == res[1][2]
    assert np.array_equal(res[0][0], res[1][0])
