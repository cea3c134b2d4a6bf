"""Replica exchange between batched jobs (smcx_batch_exchange, Sec. 2.2,
Eqs. 6-7): replicas of one lattice at a temperature ladder alternate chunks
of sweeps with exchange rounds; the ladders, accepted pairs and final
occupancies equal the oracle's (sweeps of each replica at its current
temperature, then the oracle's exchange round on the recomputed energies)."""
import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs
from tests.gpu_util import make_case, require_cuda

pytestmark = pytest.mark.gpu


def test_exchange_rounds_match_oracle(orc):
    require_cuda()
    from paper_2509_20949_gb300.batch import Batch
    kind, n, K, M = 0, (6, 6, 6), 3, 2
    ladder_T = [600.0, 660.0, 730.0, 810.0, 900.0]  # spacing ~ 1/sqrt(sites) (Sec. 2.2, Eq. 8)
    base = make_case(kind, n, K, M, seed=1, sigma=0.05, epi_seed=3, occ_seed=5)
    V = base["V"]
    R = len(ladder_T)
    reps = []
    for r in range(R):  # replicas: own initial configuration and seed
        occ = inputs.initial_occupancy(kind, n, K, 40 + r, None)
        reps.append(dict(occ=occ, seed=100 + r, t=0, T=ladder_T[r]))
    b = Batch(8, 1 << 24, 1 << 16)
    ids = [b.add(kind, n, K, rp["occ"], V, rp["T"], 10_000, seed=rp["seed"]) for rp in reps]
    ladder = list(ids)
    o_perm = np.arange(R, dtype=np.uint32)  # oracle ladder over replica indices
    descs = [orc.Desc(kind, n, K, M, seed=rp["seed"]) for rp in reps]
    total_acc = 0
    S = 4
    for rnd in range(12):
        b.run(S)
        for r, rp in enumerate(reps):  # the oracle runs each replica at its current temperature
            rp["occ"], _ = orc.sweeps(descs[r], V, rp["occ"], rp["t"], S, rp["T"])
            rp["t"] += S
        E = np.array([orc.energy(descs[r], V, rp["occ"]) for r, rp in enumerate(reps)], dtype=np.int64)
        o_perm, o_acc = orc.exchange(E, ladder_T, 77, rnd, o_perm)
        for k in range(R):
            reps[int(o_perm[k])]["T"] = ladder_T[k]
        ladder, acc = b.exchange(ladder, 77, rnd)
        assert acc == int(o_acc.sum()), rnd
        assert ladder == [ids[int(r)] for r in o_perm], rnd
        for k, jid in enumerate(ladder):
            assert b.temperature(jid) == ladder_T[k]
        total_acc += acc
    assert total_acc > 0  # the ladder is spaced so that exchanges happen
    for r, jid in enumerate(ids):
        res = b.result(jid)
        assert np.array_equal(res["occ"], reps[r]["occ"]), r
        assert res["energy"] == orc.energy(descs[r], V, reps[r]["occ"])


def test_exchange_rejects_different_systems():
    require_cuda()
    from paper_2509_20949_gb300 import SmcxError
    from paper_2509_20949_gb300.batch import Batch
    a = make_case(0, (8, 8, 8), 3, 2, seed=1)
    c = make_case(0, (8, 8, 8), 3, 2, seed=1, epi_seed=9)  # another EPI table
    b = Batch(4, 1 << 22, 1 << 14)
    ja = b.add(0, (8, 8, 8), 3, a["occ"], a["V"], 400.0, 10)
    jc = b.add(0, (8, 8, 8), 3, c["occ"], c["V"], 500.0, 10)
    with pytest.raises(SmcxError):
        b.exchange([ja, jc], 1, 0)
    with pytest.raises(SmcxError):
        b.exchange([ja, ja], 1, 0)
