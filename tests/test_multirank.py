"""The multi-rank host logic of bench.py on CPU: two gloo ranks, each with its own replica,
agree on the slowest rank's time and report all ranks' bytes over it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    w, r, local = bench.dist_setup()
    bench.dist_barrier(w)
    local_ms = 100.0 if r == 0 else 250.0           # rank 1 is the slow one
    ms_step, value = bench.aggregate(local_ms, 10, 1 << 30, w)
    q.put((r, w, local, ms_step, value))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, local, ms_step, value in out:
        assert w == 2 and local == r
        assert ms_step == pytest.approx(25.0)                     # max over ranks / steps
        assert value == pytest.approx(2 * (1 << 30) / 25e-3 / 1e9)  # both ranks' bytes
