"""Multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1) run the
whole-job aggregation; the rate uses all ranks' work over the slowest rank's
time, and every rank agrees on it."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, ms = bench.aggregate_rate(100.0 + 50.0 * rank, 1000, 4, world, "cpu")
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{value} {ms}")
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    vals = [tuple(map(float, open(tmp_path / f"r{r}.txt").read().split())) for r in range(2)]
    # slowest rank: 150 ms; work: 2 ranks x 1000 points x 5 stages x 4 steps
    for value, ms in vals:
        assert ms == pytest.approx(150.0)
        assert value == pytest.approx(2 * 1000 * 5 * 4 / 0.150)


def test_single_rank_aggregation_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.aggregate_rate(20.0, 500, 3, 1, "cpu")
    assert ms == 20.0 and value == pytest.approx(500 * 5 * 3 / 0.020)
