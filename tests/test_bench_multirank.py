"""The N > 1 path of bench.py on CPU: two gloo ranks.  Queries shard across
ranks as independent replicas, so the only exchange is the timing: every rank
must see the slowest rank's time, and the job's throughput counts the queries
of all ranks over that time."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        el_ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
        slowest = bench.max_over_ranks(el_ms, tdist, "cpu")
        value = bench.job_throughput(world, 64, 200, slowest / 1e3)
        with open(os.path.join(outdir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{slowest!r} {value!r}")
    finally:
        tdist.destroy_process_group()


def test_two_rank_timing_and_throughput(tmp_path):
    world = 2
    port = _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    res = {}
    for r in range(world):
        a, b = (tmp_path / f"rank{r}.txt").read_text().split()
        res[r] = (float(a), float(b))
    assert res[0] == res[1]                            # both ranks agree
    slowest, value = res[0]
    assert slowest == 15.0
    assert value == pytest.approx(2 * 64 * 200 / 0.015)


def _order_main(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    import time
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        def build():
            if rank == 0:
                time.sleep(0.5)                    # a slow build on rank 0
            with open(os.path.join(outdir, "order.txt"), "a") as f:
                f.write(f"{rank}\n")
            return rank
        assert bench.first_on_rank0(build, tdist, rank) == rank
    finally:
        tdist.destroy_process_group()


def test_rank0_builds_before_the_others(tmp_path):
    world = 3
    mp.spawn(_order_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    order = (tmp_path / "order.txt").read_text().split()
    assert order[0] == "0" and sorted(order) == ["0", "1", "2"]


def test_single_rank_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 64, 10, 0.5) == 1280.0
    assert bench.first_on_rank0(lambda: 7) == 7
