"""Cost-balanced sharding of the top order (gbs_range_split, host code): the
parts cover every top element, hence every order-kmax rank, exactly once, and
their entry counts differ from the mean by less than one top element's group.
Two gloo ranks on CPU each take their part, as GPUs of a sharded run would, and
the gathered parts tile the rank range."""
import os
import socket
import sys
from math import comb

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def lib_ready():
    import paper_2511_14923_gb300 as gbs
    gbs.build()
    return gbs


@pytest.mark.parametrize("M,kmax,n", [(144, 5, 8), (1024, 4, 8), (60, 5, 4), (12, 5, 7), (4096, 3, 16), (7, 2, 7)])
def test_split_tiles_and_balances(M, kmax, n):
    gbs = lib_ready()
    b = gbs.range_split(M, kmax, n)
    assert b[0] == 0 and b[-1] == M and all(x <= y for x, y in zip(b, b[1:]))
    counts = [gbs.range_entries(M, kmax, lo, hi) for lo, hi in zip(b, b[1:])]
    assert sum(counts) == comb(M, kmax)
    group = max(comb(c, kmax - 1) for c in range(M))  # entries with one top element
    assert max(counts) - comb(M, kmax) / n <= group


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import paper_2511_14923_gb300 as gbs
    dist.init_process_group("gloo")
    M, kmax = 1024, 4
    b = gbs.range_split(M, kmax, world)
    lo, hi = b[rank], b[rank + 1]
    mine = torch.tensor([comb(lo, kmax), comb(hi, kmax)], dtype=torch.int64)
    got = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(got, mine)
    q.put((rank, [g.tolist() for g in got]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_tile_the_ranks():
    lib_ready()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, parts in out:
        parts = sorted(parts)
        assert parts[0][0] == 0 and parts[-1][1] == comb(1024, 4)
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
