"""The multi-GPU path of bench.py runs independent replicas (no collective on
the data path): whole-job throughput = all ranks' solves / the slowest rank's
time.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dev = torch.device("cpu")
    bench.barrier(dist, dev)
    # Rank r solved 1000 * (r + 1) instances in 10 * (r + 1) ms.
    value, ms = bench.job_throughput(dist, 1000 * (rank + 1), 10.0 * (rank + 1), dev)
    q.put((rank, value, ms))
    dist.destroy_process_group()


def test_two_rank_replicas_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, value, ms in res:
        assert ms == 20.0                       # the slowest rank
        assert abs(value - 3000 / 0.020) < 1e-6  # all units / slowest time
