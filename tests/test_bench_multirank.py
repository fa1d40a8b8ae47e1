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


def test_oracle_legs_of_the_bench_on_small_systems():
    """The bench's CPU legs (the oracle timed as it stands) run without a GPU:
    a bounded kNN sample, a 3D sample, a whole Voronoi step and a sample of
    3D Voronoi cells."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2103_10239_gb300 import workloads as W
    w = W.uniform_system(3000, 54.0, 16, 2, input_seed=4, rule="knn", k=7, v0=0.5, eta=0.3)
    rate, m, cores, secs = bench.oracle_sample_rate(w, 0.05)
    assert rate > 0 and 32 <= m <= w.n and cores >= 1 and secs > 0
    w3 = W.uniform_system(2000, 12.6, 16, 3, input_seed=5, rule="knn", k=7, v0=0.5, eta=0.3, noise="vectorial")
    assert bench.scenario_cpu_baseline(w3, 0.05)["value"] > 0
    wv = W.uniform_system(500, 22.4, 16, 2, input_seed=6, rule="voronoi", k=0, v0=0.3, eta=0.1)
    cb = bench.scenario_cpu_baseline(wv, 0.05)
    assert cb["value"] > 0 and cb["kind"] == "oracle" and cb["cores"] == 1
    wv3 = W.voronoi_3d(n=1500)
    cb3 = bench.scenario_cpu_baseline(wv3, 0.05)
    assert cb3["value"] > 0 and cb3["kind"] == "oracle" and "1500 random particles" in cb3["sample"]
