"""Multi-GPU runs are independent replicas (one instance per rank, no data-path
collective); the whole-job throughput is the units of all ranks over the
slowest rank's time.  Checked with world_size 2 over gloo on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    # rank 0 took 2.0 s for its 10 slabs, rank 1 took 4.0 s for its 10
    value, t = bench.job_throughput(10, 2000.0 * (rank + 1), world, dist, device="cpu")
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_is_units_over_the_slowest_rank():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        value, t = out[r]
        assert t == 4000.0
        assert value == pytest.approx(20 / 4.0)


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    value, t = bench.job_throughput(7, 3500.0, 1)
    assert t == 3500.0 and value == pytest.approx(2.0)
