"""The multi-rank path of bench.py on the CPU (gloo, two ranks): each rank's
instance table is its own seeded draw from its own slice of [2^31, 2^32), so
moduli are distinct across ranks (parameter splitting, no exchange), and the
timing reduction takes the maximum over ranks."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                          WORLD_SIZE=str(world))
        sys.path.insert(0, ROOT)
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import bench
        from paper_1411_2484_gb300 import workloads
        w = dict(workloads.WORKLOADS["plain32_65536x4096x64"], instances=300)
        inst = bench.rank_instances(workloads, w, rank, world)
        everyone = [None] * world
        dist.all_gather_object(everyone, [int(x) for x in inst["n"]])
        m = bench.max_over_ranks(10.0 + rank, dist, "cpu")
        dist.destroy_process_group()
        q.put((rank, everyone, m, None))
    except Exception as exc:                        # reported to the parent
        q.put((rank, None, None, repr(exc)))


def test_two_rank_sharding_and_max_timing():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, everyone, m, err in out:
        assert err is None, err
        assert m == 10.0 + world - 1                 # the slowest rank's time
    from paper_1411_2484_gb300 import workloads
    tables = out[0][1]
    assert tables == out[1][1]                       # both ranks saw the same gather
    lo, span = 1 << 31, (1 << 31) // world
    for r, ns in enumerate(tables):
        assert len(set(ns)) == len(ns) == 300
        assert all(lo + r * span <= n < lo + (r + 1) * span for n in ns)
        assert all(workloads.is_prime(n) and workloads.is_prime((n - 1) // 2) for n in ns[:50])
    assert not set(tables[0]) & set(tables[1])
