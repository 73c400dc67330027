"""The N-GPU path of the benchmark runs N independent replicas (the path has
no exchange step); the whole job is timed by the slowest rank and its rate
counts the work of every rank. Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    # rank r takes (r + 1) seconds for its replica of 10 units
    slowest = bench.max_over_ranks(float(rank + 1), dist, "cpu")
    rate = bench.replica_rate(10.0, world, slowest)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{slowest} {rate}\n")


def test_two_gloo_ranks_take_the_slowest(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        slowest, rate = map(float, open(tmp_path / f"rank{r}.txt").read().split())
        assert slowest == 2.0
        assert rate == 10.0  # 2 replicas x 10 units / 2 s


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_rate(7.0, 1, 2.0) == 3.5
