"""Multi-rank host logic of bench.py on CPU: world size 2 over gloo.

Each rank is an independent replica: its Philox step counters must not overlap
with the other rank's, and the timing reduction must return the maximum over
ranks to every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    counters = [bench.step_counter(rank, i) for i in range(1000)]
    t = bench.max_over_ranks(1.0 + rank, dist)
    out = [None] * world
    dist.all_gather_object(out, counters)
    dist.destroy_process_group()
    q.put((rank, t, out))


def test_two_rank_replicas_disjoint_counters_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, out in res:
        assert t == 2.0                       # max of 1.0 and 2.0 on both ranks
        assert not set(out[0]) & set(out[1])  # disjoint Philox streams
