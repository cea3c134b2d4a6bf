"""z decomposition on the GPU (Sec. 2.2, lattice parallelism): plane copies
and merges of libsmcx.so, one rank equal to smcx_sweep, and two or three
ranks (processes sharing one GPU, boundary planes host-staged over gloo; no
kernel waits on another process) whose gathered lattice and summed
statistics equal the oracle's single-lattice sweeps bit for bit, for each
sweep kernel."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from tests.gpu_util import gpu_lattice, make_case, oracle_desc, require_cuda

pytestmark = pytest.mark.gpu

SCHEDULE = [(3, 1400.0, 700.0), (2, 500.0, 500.0), (1, float("inf"), float("inf"))]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_planes_copy_and_merge():
    require_cuda()
    a = gpu_lattice(make_case(0, (20, 12, 18), 4, 3, occ_seed=1))
    b = gpu_lattice(make_case(0, (20, 12, 18), 4, 3, occ_seed=2))
    occ_a, occ_b = a.occupancy(), b.occupancy()
    plane = 20 * 12 * 2

    def planes(occ, z0, nz):
        return np.concatenate([occ[((z0 + k) % 18) * plane:((z0 + k) % 18 + 1) * plane]
                               for k in range(nz)])

    z0, nz = 15, 6  # wraps the periodic seam
    before = a.get_planes(z0, nz, a.planes_buffer(nz))
    theirs = b.get_planes(z0, nz, b.planes_buffer(nz))
    a.merge_planes(z0, nz, before, before)  # nothing changed on the other side
    assert np.array_equal(a.occupancy(), occ_a)
    a.merge_planes(z0, nz, theirs, before)  # the other side changed everything
    got = a.occupancy()
    assert np.array_equal(planes(got, z0, nz), planes(occ_b, z0, nz))
    keep = np.ones(occ_a.size, bool)
    for k in range(nz):
        zz = (z0 + k) % 18
        keep[zz * plane:(zz + 1) * plane] = False
    assert np.array_equal(got[keep], occ_a[keep])
    a.put_planes(z0, nz, before)
    assert np.array_equal(a.occupancy(), occ_a)


def test_one_rank_is_the_plain_sweep():
    require_cuda()
    from paper_2509_20949_gb300.slab import SlabSweep
    case = make_case(1, (12, 10, 16), 5, 3, seed=3)
    a, b = gpu_lattice(case), gpu_lattice(case)
    s = SlabSweep(a)
    for n, t0, t1 in SCHEDULE:
        assert s.sweep(n, t0, t1) == b.sweep(n, t0, t1)
    assert np.array_equal(a.occupancy(), b.occupancy())
    assert a.running_energy() == b.running_energy() == b.energy()


def _worker(rank, world, port, case, pack_bits, kernel, q):
    import torch
    import torch.distributed as dist

    from paper_2509_20949_gb300.slab import SlabSweep
    torch.cuda.set_device(0)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lat = gpu_lattice(case, pack_bits=pack_bits, kernel=kernel)
        s = SlabSweep(lat)
        stats = [s.sweep(n, a, b) for n, a, b in SCHEDULE]
        s.gather()
        q.put((rank, lat.occupancy(), stats, lat.kernel_in_use()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind,n,K,M,pack_bits,kernel,world", [
    (0, (72, 16, 40), 5, 3, 8, 2, 2),   # BCC, tiled kernel (16x2x8 cell tiles)
    (1, (36, 12, 44), 4, 3, 8, 3, 3),   # FCC, cell kernel, three ranks
    (0, (14, 10, 27), 6, 2, 4, 0, 2),   # BCC, 4-bit storage, ragged z cells
    (1, (10, 9, 21), 3, 4, 8, 1, 2),    # FCC shells 1-4, generic kernel, ragged
])
def test_ranks_reproduce_the_single_lattice(orc, kind, n, K, M, pack_bits, kernel, world):
    require_cuda()
    case = make_case(kind, n, K, M, seed=7, epi_seed=8, occ_seed=9)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, pack_bits, kernel, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # the oracle's single-lattice sweeps over the same schedule
    d = oracle_desc(orc, case)
    occ, t0, want = case["occ"], 0, []
    for nsw, a, b in SCHEDULE:
        occ, st = orc.sweeps(d, case["V"], occ, t0, nsw, a, b)
        t0 += nsw
        want.append({k: int(st[k].sum()) for k in ("attempts", "unlike", "accepted", "sum_dE")})
    for rank, r_occ, stats, kin in res:
        if kernel:
            assert kin[0] == kernel
        assert stats == want, rank
        assert np.array_equal(r_occ, occ), rank
