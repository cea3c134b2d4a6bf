"""Whole colour phases of the 1.07e9-site lattices against the oracle.

One colour phase of the benchmark lattice (BCC 812^3 x 2, 8,365,427 link
cells, 133.8M trials) runs on the GPU in the kernel the benchmark times (the
online choice, after its tuning sweeps); the oracle replays every link cell
of the same phase from the same starting bits, with the cells shared out
over the host cores (cells of one colour never interact, Sec. 2.2, so this
is the sequential result).  The whole lattice must agree byte for byte --
written sites, and the sites no cell may touch -- and so must the phase's
attempts, unlike pairs, accepted swaps and sum of dE.  The same for the
4-bit packed storage and for the paper's production lattice (FCC 672 x 630
x 630 x 4, ragged link cells in y and z, shells 1-4)."""
import numpy as np
import pytest

from tests.gpu_util import colour_cells, gpu_lattice, make_case, oracle_desc, require_cuda

pytestmark = pytest.mark.gpu

TILED = 2


def _anneal_T(w, t):
    return w["T_first"] + (w["T_last"] - w["T_first"]) * t / (w["sweeps"] - 1)


def _whole_phase(orc, name, pack_bits, warm_sweeps, colour):
    torch = require_cuda()
    from paper_2509_20949_gb300 import inputs
    w = inputs.workload(name)
    case = make_case(w["kind"], w["n"], w["K"], w["M"], seed=w["seed"], sigma=w["sigma"],
                     epi_seed=w["epi_seed"], occ_seed=w["occ_seed"], fractions=w["fractions"])
    lat = gpu_lattice(case, pack_bits=pack_bits)
    d = oracle_desc(orc, case)
    # the first sweeps also run the online kernel choice
    lat.sweep(warm_sweeps, _anneal_T(w, 0), _anneal_T(w, warm_sweeps - 1))
    assert lat.kernel_in_use()[0] == TILED
    t = lat.sweep_counter
    T = _anneal_T(w, t)
    before = lat.occupancy()
    g = lat.run_colour(colour, T)
    after = lat.occupancy()
    E_run = lat.running_energy()
    E_gpu = lat.energy()
    lat.close()
    del lat
    torch.cuda.empty_cache()
    cids = colour_cells(orc, d, colour)
    o_occ, o = orc.phase_cells_par(d, case["V"], before, t, T, colour, cids, inplace=False)
    assert (g["attempts"], g["unlike"], g["accepted"], g["sum_dE"]) == \
        (int(o["attempts"]), int(o["unlike"]), int(o["accepted"]), int(o["sum_dE"]))
    diff = np.flatnonzero(after != o_occ)
    assert diff.size == 0, f"{diff.size} sites differ, first {diff[:8]}"
    assert int(o["accepted"]) > 0 and np.count_nonzero(before != after) > 0
    # incremental energy (base taken at set_epi) = full recompute on the GPU
    assert E_run == E_gpu


def test_bcc812_whole_phase_matches_oracle(orc):
    _whole_phase(orc, "bcc812_k5", 8, 2, 5)


def test_bcc812_packed_whole_phase_matches_oracle(orc):
    _whole_phase(orc, "bcc812_k5", 4, 2, 2)


def test_fcc672_whole_phase_matches_oracle(orc):
    _whole_phase(orc, "fcc672_k5", 8, 2, 6)
