"""bench.py's multi-rank paths (independent cells per GPU, no data-path
collective) on gloo ranks on CPU: the max of the device times and the sum of
the particle-steps, and the batch's rank slices."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms, ps = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), dist)
    q.put((rank, ms, ps))
    dist.destroy_process_group()


def test_two_rank_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, ps in out:
        assert ms == 15.0 and ps == 3000.0


def _slice_rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from paper_2609_15043_b300 import workloads
    mine = bench.batch_slice(workloads.batch_cells(), rank, ws)
    got = [None] * ws
    dist.all_gather_object(got, [repr(c) for c in mine])
    q.put((rank, got))
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_batch_slices_cover_the_batch(ws):
    """Every cell of the 32-cell batch is advanced by exactly one rank, with the
    configuration (grid, population, seed) it has in the unsliced batch, so
    each rank's cells are the same independent problems as in one process."""
    sys.path.insert(0, ROOT)
    from paper_2609_15043_b300 import workloads
    full = [repr(c) for c in workloads.batch_cells()]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slice_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got in out:
        union = [c for sl in got for c in sl]
        assert sorted(union) == sorted(full)
        assert len(union) == len(full) == len(set(full))
        for r, sl in enumerate(got):
            assert sl == full[r::ws]
