"""The multi-process path of bench.py on the CPU: two `gloo` ranks, as
torchrun launches them (one independent replica per rank, no collective on
the data path; only the timings are combined)."""
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as td
    import bench
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed 1000 (r + 1) particle-steps in 0.5 + r seconds
        units, secs = bench.reduce_job(td, 1000 * (rank + 1), 0.5 + rank, "cpu")
        q.put((rank, units, secs))
    finally:
        td.destroy_process_group()


def test_two_ranks_sum_the_work_and_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, units, secs in got:
        assert units == 3000.0  # every rank's units count
        assert secs == 1.5  # the slowest rank sets the time


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_job(None, 123, 0.25, "cpu") == (123.0, 0.25)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    # any rank other than 0 returns at once, without touching the oracle
    assert bench.run_reference(None, 1, 2) is None
