"""The bench's multi-GPU form runs independent replicas (the layout has no
shard): whole-job throughput = units of all ranks / slowest rank's time.
Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 250.0][rank]
    value, max_ms = bench.replica_throughput(local_ms, 1e9, dist, "cpu")
    q.put((rank, value, max_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
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
    for rank, value, max_ms in out:
        assert max_ms == 250.0
        assert value == pytest.approx(2 * 1e9 / 0.25)


def test_replica_throughput_single_process():
    import bench
    assert bench.replica_throughput(500.0, 1e9) == (2e9, 500.0)
