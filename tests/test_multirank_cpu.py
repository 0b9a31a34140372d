"""The N > 1 path of bench.py on CPU: gloo, world_size 2.  Each rank solves
its own transforms (replicas); the job's time is the max over ranks and the
value counts every rank's coefficients."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_time = 1.0 + rank          # rank 1 is the slower one
    t = bench.max_over_ranks(local_time)
    v = bench.whole_job_value(8008, 10, world, t)
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks_and_value_counts_all_ranks():
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
    for rank, t, v in res:
        assert t == 2.0
        assert v == pytest.approx(2 * 8008 * 10 / 2.0)
