"""Continuous-batching server: jobs arriving while others run are admitted
as slots and arena space free up, and every job's result is bit-identical to
the same lattice run alone."""
import numpy as np
import pytest

from paper_2509_20949_gb300 import inputs
from tests.gpu_util import require_cuda

pytestmark = pytest.mark.gpu


def _trace(count, seed):
    rng = np.random.default_rng(seed)
    jobs = []
    t = 0.0
    for j in range(count):
        t += rng.exponential(0.01)
        kind = int(rng.integers(0, 2))
        n = int(rng.integers(4, 20))
        K = int(rng.integers(3, 7))
        fr = inputs.dirichlet_fractions(K, 5.0, 40 + j) if rng.uniform() < 0.5 else None
        jobs.append(dict(arrival_s=t, kind=kind, n=(n, n, n), K=K, M=3,
                         V=inputs.epi_table(3, K, 0.02, 500 + j),
                         occ=inputs.initial_occupancy(kind, (n, n, n), K, 600 + j, fr),
                         T=float(rng.uniform(300, 1500)), sweeps=int(rng.integers(5, 60)),
                         seed=700 + j))
    return jobs


def _alone(job):
    from paper_2509_20949_gb300.lattice import Lattice
    lat = Lattice(job["kind"], job["n"], job["K"], job["occ"], seed=job["seed"])
    lat.set_epi(job["V"])
    st = lat.sweep(job["sweeps"], job["T"])
    return lat.occupancy(), st, lat.running_energy()


def test_served_results_equal_alone_runs():
    require_cuda()
    from paper_2509_20949_gb300.batch import Batch
    from paper_2509_20949_gb300.server import Server
    jobs = _trace(24, 3)
    biggest = max(Batch.job_bytes(j["kind"], j["n"], j["K"]) for j in jobs)
    # a budget of ~3 of the largest lattices and 6 slots: admission has to wait
    srv = Server(budget_bytes=3 * biggest, max_jobs=6, chunk_sweeps=8, transfer_bytes=1 << 20)
    m = srv.run_trace(jobs, deadline_s=300)
    assert m["completed"] == len(jobs) and m["completed_fraction"] == 1.0
    assert srv.chunks > 1 and m["p99_latency_s"] >= m["p50_latency_s"] > 0
    for ticket, job in enumerate(jobs):
        r = srv.done[ticket]
        occ, st, E = _alone(job)
        assert np.array_equal(r["occ"], occ), ticket
        assert r["stats"] == st and r["energy"] == E and r["sweeps"] == job["sweeps"]


def test_launch_wait_overlap_admission_and_readback():
    """Chunks launched without waiting (smcx_batch_launch / smcx_batch_wait):
    while one runs, a new job is admitted through the side stream and a job
    finished by an earlier chunk is read back; every job still ends in the
    bits of its run alone."""
    require_cuda()
    from paper_2509_20949_gb300.batch import Batch
    jobs = _trace(6, 9)
    jobs[0]["sweeps"] = 8                       # finishes in the first chunks
    for j in jobs[1:]:
        j["sweeps"] = max(j["sweeps"], 40)
    transfer = max(inputs.n_sites(j["kind"], j["n"]) for j in jobs)
    heap = sum(Batch.job_bytes(j["kind"], j["n"], j["K"]) for j in jobs)
    b = Batch(8, Batch.control_bytes(8, transfer) + heap + (1 << 20), transfer)
    # slot ids are reused after remove: keep the slot -> job map current
    slot_job = {b.add(j["kind"], j["n"], j["K"], j["occ"], j["V"], j["T"], j["sweeps"],
                      seed=j["seed"]): k for k, j in enumerate(jobs[:4])}
    results, launched_while_busy = {}, 0
    late = {k: j for k, j in enumerate(jobs) if k >= 4}
    for _ in range(400):
        b.launch(4)
        if late and b.tuning()["tuned"]:
            k, j = late.popitem()               # admitted while the chunk runs
            slot_job[b.add(j["kind"], j["n"], j["K"], j["occ"], j["V"], j["T"], j["sweeps"],
                           seed=j["seed"])] = k
            launched_while_busy += 1
        for jid in b.poll():                    # finished by an earlier chunk
            results[slot_job.pop(jid)] = b.result(jid)
            b.remove(jid)
        b.wait()
        if len(results) == len(jobs):
            break
    for jid in b.poll():
        results[slot_job.pop(jid)] = b.result(jid)
    assert launched_while_busy == 2 and len(results) == len(jobs)
    for k, job in enumerate(jobs):
        occ, st, E = _alone(job)
        r = results[k]
        assert np.array_equal(r["occ"], occ), k
        assert r["stats"] == st and r["energy"] == E and r["sweeps"] == job["sweeps"], k
    b.close()
