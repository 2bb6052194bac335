"""The N > 1 path of bench.py (independent replicas, no data-path collective):
the job time is the slowest rank's and the value counts every rank's table.
Two gloo ranks on CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    r, w, d = bench.dist_init(world, backend="gloo")
    ms = [12.0, 15.5][r]
    tot = bench.max_over_ranks(ms, d, "cpu")
    val = bench.replica_value(1000, 4, w, tot)
    q.put((r, w, tot, val))
    d.barrier()
    d.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, tot, val in out:
        assert w == 2 and tot == 15.5
        assert val == pytest.approx(1000 * 4 * 2 / 15.5e-3)
