"""Multi-rank plumbing of bench.py on CPU (gloo, world size 2): the path runs
as independent replicas, so the only cross-rank step is the barrier and the
max-over-ranks timing that rank 0 reports."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench.dist_setup()
    assert (ws, r) == (world, rank)
    bench.barrier(ws)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, ws)
    out[rank] = t
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()  # no fork of a multi-threaded process
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == 15.0
