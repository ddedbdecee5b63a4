"""The multi-rank path of the benchmark on CPU: world size 2 over gloo.

Each rank takes its own independent case (no data-path collective) and only
the timings are combined: max of the times, sum of the work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2301_09349_gb300 import replicas
    c = replicas.case_for_rank(rank, world, n=32)
    ms = 10.0 + rank            # rank 1 is the slower one
    e2e = 20.0 - rank
    out = replicas.reduce_timings(dist, torch.device("cpu"), ms, e2e, float(c.grid.ncells),
                                  float(len(c.X)))
    q.put((rank, c.name, out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_distinct_cases_and_combine_timings():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, name0, out0), (r1, name1, out1) = res
    assert name0 != name1
    assert out0 == out1
    ms, e2e, cells, markers = out0
    assert ms == 11.0 and e2e == 20.0
    assert cells == 2 * 32 ** 3


def test_single_rank_is_identity():
    from paper_2301_09349_gb300 import replicas
    assert replicas.reduce_timings(None, None, 1.0, 2.0, 3.0, 4.0) == (1.0, 2.0, 3.0, 4.0)
    c = replicas.case_for_rank(0, 1, n=32)
    assert c.grid.Mach == 0.3
