"""The z decomposition's host protocol (SlabSweep: half-sweep boundary merges,
plane moves between sweeps, gather) on gloo ranks on the CPU: each rank's
whole-lattice copy is an oracle colour-phase replay, and after the sweeps the
gathered lattice and the summed statistics equal the oracle's single-lattice
sweeps bit for bit (Sec. 2.2, lattice parallelism) -- with the boundary
exchange overlapping the interior planes' sweep (Sec. 3.1) and without."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2509_20949_gb300 import inputs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case(kind, n, K, M, seed):
    V = inputs.epi_table(M, K, 0.03, seed + 1)
    occ = inputs.initial_occupancy(kind, n, K, seed + 2)
    return dict(kind=kind, n=tuple(n), K=K, M=M, seed=seed, flags=0, min_cell=0, V=V, occ=occ)


SCHEDULE = [(3, 1500.0, 900.0), (2, 600.0, 600.0), (1, float("inf"), float("inf"))]


def _worker(rank, world, port, case, q, overlap=True):
    import torch.distributed as dist

    import oracle
    from paper_2509_20949_gb300.slab import SlabSweep
    from tests.slab_engine import OracleRankLattice

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lat = OracleRankLattice(oracle, case)
        s = SlabSweep(lat, overlap=overlap)
        stats = [s.sweep(n, a, b) for n, a, b in SCHEDULE]
        s.gather()
        q.put((rank, lat.occ.copy(), stats, lat.sweep_counter))
    finally:
        dist.destroy_process_group()


def _run(case, world, overlap=True):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q, overlap))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res, key=lambda r: r[0])


@pytest.mark.parametrize("kind,n,K,M,world,overlap", [
    (0, (6, 6, 16), 4, 2, 2, True),     # BCC, uniform cells
    (0, (6, 6, 16), 4, 2, 2, False),
    (0, (6, 5, 13), 3, 3, 3, True),     # BCC, ragged z cells, three ranks
    (1, (4, 4, 12), 3, 4, 2, True),     # FCC, shells 1-4
    (0, (5, 4, 17), 3, 2, 4, True),     # four ranks: distinct neighbours on both sides, ragged
    (0, (5, 4, 17), 3, 2, 4, False),
    (0, (4, 4, 40), 3, 3, 2, True),     # ranks of 10 cell planes: interior planes overlap the exchange
    (0, (4, 4, 36), 3, 4, 2, True),     # shells 1-4 (edge 3): interior planes overlap the exchange
])
def test_ranks_reproduce_the_single_lattice_sweeps(orc, kind, n, K, M, world, overlap):
    case = _case(kind, n, K, M, seed=40 + world)
    res = _run(case, world, overlap)
    d = orc.Desc(kind, n, K, M, seed=case["seed"])
    occ = case["occ"].copy()
    t = 0
    want = []
    for nsw, a, b in SCHEDULE:
        occ, per = orc.sweeps(d, case["V"], occ, t, nsw, a, b)
        t += nsw
        want.append({k: sum(p[k] for p in per) for k in ("attempts", "unlike", "accepted", "sum_dE")})
    for rank, r_occ, stats, tc in res:
        assert tc == t
        assert np.array_equal(r_occ, occ), rank
        assert stats == want, rank
