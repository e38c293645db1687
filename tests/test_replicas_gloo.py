"""Host logic of the multi-GPU form (replicas, no data-path collective) on
CPU: two gloo ranks reduce their step times to the max over ranks, and the
whole-job throughput counts every rank's units over that time."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    assert bench.dist_env() == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.replica_time(10.0 * (rank + 1), world)
        value = bench.job_throughput(1000.0, world, ms)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{ms} {value}\n")
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    for r in range(world):
        ms, value = map(float, (tmp_path / f"r{r}.txt").read_text().split())
        assert ms == pytest.approx(20.0)
        assert value == pytest.approx(2 * 1000.0 / 0.020)


def test_single_process_needs_no_group():
    import bench
    assert bench.replica_time(3.5, 1) == 3.5
    assert bench.job_throughput(100.0, 1, 2.0) == pytest.approx(5e4)
