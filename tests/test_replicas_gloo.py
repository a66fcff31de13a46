"""The N > 1 path of bench.py on CPU: world_size-2 gloo process groups
(replicas only, no data-path collective). The job time is the slowest
rank's and the throughput counts every rank's points; the reference arm
runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, local_ms, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms, val = bench.replica_throughput(local_ms[rank], 1_000_000, dist)
    q.put((rank, ms, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    local = [2.0, 5.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, local, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, val in got:
        assert ms == 5.0
        assert val == pytest.approx(2 * 1_000_000 / 5e-3 / 1e9)


def test_single_process_has_no_group():
    import bench
    ms, val = bench.replica_throughput(4.0, 2_000_000)
    assert ms == 4.0 and val == pytest.approx(2_000_000 / 4e-3 / 1e9)
