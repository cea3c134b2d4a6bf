"""Host-side logic of the multi-GPU benchmark (independent replicas, one
per rank): world-size-2 gloo process groups on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mx = bench.max_over_ranks(10.0 + 5.0 * rank)
    seed = bench.replica_seed(7, rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, seed))


def test_max_over_ranks_and_replica_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [15.0, 15.0]
    assert [r[2] for r in res] == [7, 8]


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
