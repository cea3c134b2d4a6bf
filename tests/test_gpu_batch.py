"""Batched execution (smcx_batch_*): every job's trajectory equals the same
lattice run alone through smcx_sweep, and the oracle, bit for bit; jobs can
join and leave between chunks; admission respects the arena budget."""
import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs
from tests.gpu_util import make_case, require_cuda

pytestmark = pytest.mark.gpu


def _jobs(seed, count, nmin=4, nmax=14):
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(count):
        kind = int(rng.integers(0, 2))
        n = tuple(int(v) for v in rng.integers(nmin, nmax + 1, 3))
        K = int(rng.integers(2, 7))
        M = int(rng.integers(2, 5))
        T = float(rng.choice([0.0, 300.0 + 1200.0 * rng.uniform(), float("inf")], p=[0.1, 0.8, 0.1]))
        case = make_case(kind, n, K, M, seed=100 + j, sigma=0.03, epi_seed=200 + j, occ_seed=300 + j)
        case.update(T=T, sweeps=int(rng.integers(1, 25)))
        jobs.append(case)
    return jobs


def _alone(case):
    from paper_2509_20949_gb300.lattice import Lattice
    lat = Lattice(case["kind"], case["n"], case["K"], case["occ"], seed=case["seed"])
    lat.set_epi(case["V"])
    st = lat.sweep(case["sweeps"], case["T"])
    return lat.occupancy(), st, lat.running_energy()


def _batch(max_jobs=64, arena=1 << 26, transfer=1 << 20):
    from paper_2509_20949_gb300.batch import Batch
    return Batch(max_jobs, arena, transfer)


def _add(b, case):
    return b.add(case["kind"], case["n"], case["K"], case["occ"], case["V"], case["T"],
                 case["sweeps"], seed=case["seed"])


def test_batch_matches_alone_and_oracle(orc):
    require_cuda()
    jobs = _jobs(1, 14)
    b = _batch()
    ids = [_add(b, c) for c in jobs]
    done = set()
    for _ in range(40):
        b.run(6)
        done |= set(b.poll())
        if len(done) == len(jobs):
            break
    assert done == set(ids)
    for jid, c in zip(ids, jobs):
        r = b.result(jid)
        occ, st, E = _alone(c)
        assert np.array_equal(r["occ"], occ), jid
        assert r["stats"] == st and r["energy"] == E and r["sweeps"] == c["sweeps"]
    # the oracle for a few of them
    for jid, c in list(zip(ids, jobs))[:4]:
        d = orc.Desc(c["kind"], c["n"], c["K"], c["M"], seed=c["seed"])
        o_occ, _ = orc.sweeps(d, c["V"], c["occ"], 0, c["sweeps"], c["T"])
        assert np.array_equal(b.result(jid)["occ"], o_occ)


def test_jobs_join_and_leave_between_chunks():
    require_cuda()
    jobs = _jobs(2, 12)
    b = _batch(max_jobs=5)
    pending = list(range(len(jobs)))
    running = {}
    finished = {}
    chunks = 0
    while pending or running:
        while pending and b.info()["free_slots"] > 0:
            k = pending.pop(0)
            running[_add(b, jobs[k])] = k
        b.run(4)
        chunks += 1
        for jid in b.poll():
            k = running.pop(jid)
            finished[k] = b.result(jid)
            b.remove(jid)
        assert chunks < 200
    for k, c in enumerate(jobs):
        occ, st, E = _alone(c)
        assert np.array_equal(finished[k]["occ"], occ), k
        assert finished[k]["stats"] == st and finished[k]["energy"] == E


def test_admission_budget():
    require_cuda()
    from paper_2509_20949_gb300 import SmcxError
    from paper_2509_20949_gb300.batch import Batch
    case = make_case(0, (16, 16, 16), 4, 3, seed=1)
    case.update(T=800.0, sweeps=3)
    per_job = Batch.job_bytes(0, (16, 16, 16), 4)
    ctrl = Batch.control_bytes(8, 1 << 16)
    b = Batch(8, ctrl + 2 * per_job, 1 << 16)
    a = _add(b, case)
    _add(b, case)
    assert b.try_add(case["kind"], case["n"], case["K"], case["occ"], case["V"], 800.0, 3) is None
    b.remove(a)
    assert b.info()["free_bytes"] >= per_job
    _add(b, case)
    with pytest.raises(SmcxError):
        b.add(0, (3, 4, 4), 3, np.zeros(96, np.uint8), inputs.epi_table(2, 3, 0.02, 0), 500.0, 1)


def _mixed_jobs():
    """Small jobs (one item per phase) next to larger ragged ones (many items
    per phase), so that phases of one job span several warps."""
    jobs = _jobs(3, 8, nmin=4, nmax=12)
    for j, (kind, n, K, M) in enumerate([(1, (26, 22, 30), 5, 3), (0, (40, 37, 34), 6, 4),
                                          (0, (33, 48, 20), 4, 2)]):
        case = make_case(kind, n, K, M, seed=500 + j, sigma=0.03, epi_seed=600 + j, occ_seed=700 + j)
        case.update(T=700.0 + 300.0 * j, sweeps=9 + j)
        jobs.append(case)
    return jobs


def _run_all(b, jobs, chunk):
    ids = [_add(b, c) for c in jobs]
    done = set()
    for _ in range(100):
        b.run(chunk)
        done |= set(b.poll())
        if len(done) == len(jobs):
            break
    assert done == set(ids)
    return [b.result(j) for j in ids]


def test_every_tuning_choice_gives_the_same_bits():
    """Work-item shape, schedule and register budget change only speed."""
    require_cuda()
    from paper_2509_20949_gb300.batch import Batch
    jobs = _mixed_jobs()
    alone = [_alone(c) for c in jobs]
    for tile in range(4):
        assert np.prod(Batch.tile_shape(tile)) == 32
        for sched in range(2):
            for occ in range(2):
                b = _batch(max_jobs=16, arena=1 << 27)
                b.set_option(Batch.OPT_TILE, tile)
                b.set_option(Batch.OPT_SCHEDULE, sched)
                b.set_option(Batch.OPT_OCCUPANCY, occ)
                res = _run_all(b, jobs, 5)
                assert b.tuning() == dict(tile=tile, schedule=sched, occupancy=occ, tuned=True)
                for k, (r, (occ_a, st, E)) in enumerate(zip(res, alone)):
                    assert np.array_equal(r["occ"], occ_a), (tile, sched, occ, k)
                    assert r["stats"] == st and r["energy"] == E, (tile, sched, occ, k)
                if sched == 1:
                    assert b.queue_stats()["waited_items"] == 0  # no device-side waits
                b.close()


def test_online_tuning_converges_without_changing_results():
    require_cuda()
    jobs = _mixed_jobs()
    for c in jobs:
        c["sweeps"] = 30
    b = _batch(max_jobs=16, arena=1 << 27)
    assert b.tuning()["tuned"] is False
    res = _run_all(b, jobs, 30)
    t = b.tuning()
    assert t["tuned"] and 0 <= t["tile"] < 4 and 0 <= t["schedule"] < 2 and 0 <= t["occupancy"] < 2
    for k, (r, c) in enumerate(zip(res, jobs)):
        occ_a, st, E = _alone(c)
        assert np.array_equal(r["occ"], occ_a), k
        assert r["stats"] == st and r["energy"] == E and r["sweeps"] == 30


def test_persistent_plan_with_many_jobs_and_segments():
    """The persistent schedule's plan over 400 jobs of uneven size (many
    segments per warp for the small ones, one job spread over many warps):
    the jobs end as they do alone, including jobs that stop in the middle of
    a chunk."""
    require_cuda()
    from paper_2509_20949_gb300.batch import Batch
    jobs = _jobs(9, 399, nmin=4, nmax=9)
    big = make_case(1, (44, 40, 36), 5, 3, seed=900, sigma=0.03, epi_seed=901, occ_seed=902)
    big.update(T=900.0, sweeps=7)
    jobs.append(big)
    b = _batch(max_jobs=400, arena=1 << 28, transfer=1 << 21)
    b.set_option(Batch.OPT_SCHEDULE, 0)
    b.set_option(Batch.OPT_TILE, 0)
    ids = [_add(b, c) for c in jobs]
    done = set()
    for _ in range(20):
        b.run(5)
        done |= set(b.poll())
        if len(done) == len(jobs):
            break
    assert done == set(ids)
    assert b.tuning()["schedule"] == 0
    for k in list(range(0, len(jobs), 37)) + [len(jobs) - 1]:
        r = b.result(ids[k])
        occ, st, E = _alone(jobs[k])
        assert np.array_equal(r["occ"], occ), k
        assert r["stats"] == st and r["energy"] == E, k
    b.close()
