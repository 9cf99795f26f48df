"""The N > 1 path of the throughput measurement on the CPU: two gloo ranks (replicas, no data-path
collective) agree on the slowest rank's time, compute the whole-job rate from it, and only rank 0
runs the CPU-oracle reference arm."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(1.5 + rank)            # rank r took 1.5 + r time units
    rate = bench.whole_job_rate(6e12, slowest, world)     # same work on every rank
    ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "gpus": world})(), rank) if rank else None
    tdist.barrier()
    tdist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write("%r %r %r\n" % (slowest, rate, ref))


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        slowest, rate, ref = open(tmp_path / ("rank%d.txt" % r)).read().split(" ", 2)
        assert float(slowest) == 2.5                       # the max over ranks, on every rank
        assert abs(float(rate) - world * 6e12 / 2.5 / 1e12) < 1e-9
        assert ref.strip() == "None"                       # rank 1 skips the reference arm
