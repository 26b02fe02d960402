"""Multi-rank path of bench.py on CPU with gloo (world size 2).

With N GPUs the benchmark runs N independent replicas (no collective on the data
path); the ranks only meet at the timing barrier and the max-reduction of the elapsed
time, and the whole-job value is all ranks' solves over the slowest rank's time.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    d = bench.Dist()
    d.init("gloo")
    d.barrier()
    ms = 10.0 + 5.0 * rank                      # this rank's timed region
    slowest = d.max(ms)
    steps = 4
    value = d.world * steps / (slowest / 1e3)   # whole-job solves/s
    d.barrier()
    q.put((rank, slowest, value))
    d.done()


def test_replicas_take_max_over_ranks():
    import torch.multiprocessing as mp

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
    assert [o[1] for o in out] == [15.0, 15.0]
    assert all(o[2] == pytest.approx(2 * 4 / 0.015) for o in out)
