"""Multi-rank host logic of bench.py on CPU: two gloo ranks (spawned
processes on 127.0.0.1), each timing a different replica; the job time is the
slowest rank's and the job MLUPS counts the lattice updates of all ranks."""
from __future__ import annotations

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        assert (r, w, lr) == (rank, world, rank)
        seconds = [1.25, 2.5, 0.75, 1.0][rank]
        slowest = bench.max_over_ranks(seconds, world)
        value = bench.aggregate_mlups(16_000_000, 100, world, slowest)
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r\n" % (slowest, value))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_and_job_mlups(tmp_path, world):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    expect_t = max([1.25, 2.5, 0.75, 1.0][:world])
    expect_v = 16_000_000 * world * 100 / expect_t / 1e6
    for rank in range(world):
        slowest, value = map(float, (tmp_path / ("rank%d.txt" % rank)).read_text().split())
        assert slowest == expect_t
        assert value == pytest.approx(expect_v, rel=1e-12)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_mlups(1000, 10, 1, 2.0) == pytest.approx(1000 * 10 / 2.0 / 1e6)
