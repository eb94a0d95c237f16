"""Multi-rank bench logic on CPU (gloo, world_size 2): every rank gets its own disjoint
slice of DE candidates (weak scaling, no data-path collective) and the reported time is
the maximum over ranks."""
import os
import socket
import sys

import pytest
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
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pop = bench._population(rank)
        names = [p.name for p in pop]
        t = bench._max_over_ranks(10.0 + rank)
        q.put((rank, names, t))
    finally:
        dist.destroy_process_group()


def test_population_shards_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (r0, n0, t0), (r1, n1, t1) = out
    assert len(n0) == len(n1) == 64
    assert not set(n0) & set(n1)
    assert n0[0] == "de000" and n1[0] == "de064"
    assert t0 == t1 == 11.0
