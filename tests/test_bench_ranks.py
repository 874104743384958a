"""The bench's multi-rank path on CPU: two or four gloo ranks (replicas, no data-path
collective) agree on the max time and the summed work, as bench.py reports them."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    t = bench.max_over_ranks(w, 1.0 + rank, torch.device("cpu"))
    n = bench.sum_over_ranks(w, 10.0 * (rank + 1), torch.device("cpu"))
    q.put((rank, t, n))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_rank_max_and_sum(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert [g[1] for g in got] == [float(world)] * world                       # max over ranks
    assert [g[2] for g in got] == [5.0 * world * (world + 1)] * world          # work summed over ranks
