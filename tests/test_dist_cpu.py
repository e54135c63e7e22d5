"""The multi-GPU path is replicas only (blocks and files are independent
units; no exchange step): each rank decodes its own copy of the workload and
rank 0 reports the bytes of all ranks over the slowest rank's time.  This
checks the host-side pieces of that path with two gloo ranks on the CPU:
the barrier, the max of the ranks' times and the sum of their bytes."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, local, dist = bench._dist_init(None)
    bench._barrier(dist)
    t = bench._max_over_ranks(dist, 10.0 + rank)
    b = bench._sum_over_ranks(dist, 1000.0 * (rank + 1))
    q.put((r, w, t, b))
    dist.destroy_process_group()


@pytest.mark.timeout(120, method="thread")
def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == 11.0 for r in res)       # max over ranks
    assert all(r[3] == 3000.0 for r in res)     # sum of bytes over ranks
