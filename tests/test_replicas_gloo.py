"""The multi-GPU path runs independent replicas (no data-path collective):
the whole-job throughput is world x units / the slowest rank's step time.
Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    step_ms = [2.0, 5.0][rank]          # rank 1 is the slow replica
    value, worst = bench.replica_throughput(step_ms, 5000, world)
    dist.barrier()
    out[rank] = (value, worst)
    dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        value, worst = out[r]
        assert worst == 5.0
        assert abs(value - 2 * 5000 / 5e-3) < 1e-6


def test_single_rank_needs_no_process_group():
    import bench
    value, worst = bench.replica_throughput(4.0, 1000, 1)
    assert worst == 4.0 and abs(value - 1000 / 4e-3) < 1e-9
