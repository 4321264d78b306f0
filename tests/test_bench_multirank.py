"""The multi-rank timing path of bench.py on CPU (gloo, world size 2).

Each rank runs an independent replica; the whole-job rate is all ranks'
steps over the slowest rank's time.  No collective touches the data path.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    class A:
        pass
    r, w = bench.dist_setup(A())
    local_ms = 100.0 * (rank + 1)  # rank 1 is the slowest
    value, tmax = bench.job_throughput(local_ms, 10, w)
    out.put((r, w, value, tmax))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_job_throughput_takes_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, value, tmax in res:
        assert w == 2
        assert tmax == 200.0
        assert abs(value - 2 * 10 / 0.2) < 1e-9
