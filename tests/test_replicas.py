"""The N > 1 bench path (independent replicas, no data-path collective):
two gloo ranks on CPU check that the whole-job throughput is all sweeps over
the slowest replica's time."""
import os
import socket

import pytest
import torch.distributed as tdist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)            # rank 1 is the slow replica
    value, slowest = bench.replica_throughput(world, 20, local_ms)
    tdist.barrier()
    q.put((rank, value, slowest))
    tdist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
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
    for rank, value, slowest in out:
        assert slowest == 200.0
        assert abs(value - 2 * 20 / 0.2) < 1e-9
