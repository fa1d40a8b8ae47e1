"""Batched replicas: one launch per kernel covers all replicas, and every
replica is bit-identical to the same system run on its own."""
import numpy as np
import pytest

from paper_2103_10239_gb300 import vk
from paper_2103_10239_gb300 import workloads as W
from parity import check_step

pytestmark = pytest.mark.gpu


def test_batch_equals_single_runs():
    ws = W.replica_batch(n_rep=12, sizes=[1024, 1500, 3000, 1100, 65536, 2047, 4096, 1025, 9000,
                                          1024, 20000, 1300])
    with vk.batch_from_workloads(ws) as sim:
        sim.set_graph_steps(5)
        sim.step(20)
        batch = [sim.state(r) for r in range(len(ws))]
        phis = [sim.order_parameter(r) for r in range(len(ws))]
    for r, w in enumerate(ws):
        pos, d, _, t = batch[r]
        assert t == 20
        assert phis[r].shape[0] == 20
    # the replica index enters the noise counter, so replica r of a batch of
    # r+1 replicas must reproduce replica r of the full batch bit for bit
    for r in (0, 4, 7, 11):
        with vk.batch_from_workloads(ws[: r + 1]) as sim:
            sim.step(20)
            pos, d, _, _ = sim.state(r)
        assert np.array_equal(pos, batch[r][0])
        assert np.array_equal(d, batch[r][1])
    # and a single system created on its own with replica_offset = r (its own
    # grid, its own launches) reproduces it too
    for r in (3, 4, 10):
        with vk.from_workload(ws[r], replica_offset=r) as sim:
            sim.step(20)
            pos, d, _, t = sim.state()
        assert t == 20
        assert np.array_equal(pos, batch[r][0])
        assert np.array_equal(d, batch[r][1])


def test_batch_teacher_forced_parity():
    ws = W.replica_batch(n_rep=6, sizes=[1024, 2000, 5000, 1200, 3000, 1500])
    with vk.batch_from_workloads(ws) as sim:
        for r in (0, 2, 5):
            check_step(sim, ws[r], "knn", replica=r)


def test_full_replica_batch_runs():
    ws = W.replica_batch()
    with vk.batch_from_workloads(ws) as sim:
        sim.set_graph_steps(10)
        sim.step(20)
        sim.sync()
        phi = sim.order_parameter(511)
        assert phi.shape[0] == 20 and np.all((phi >= 0) & (phi <= 1))
        check_step(sim, ws[300], "knn", replica=300)


def test_voronoi_batch_equals_single_runs():
    """The Voronoi rule in a batch (seeds, heavy-cell flags and the cost-
    grouped visiting order are all per replica): every replica equals the
    same system alone, and the lists of each match the oracle."""
    import oracle
    ws = W.replica_batch(n_rep=5, sizes=[1024, 3000, 1500, 700, 2500])
    for w in ws:
        w.rule = "voronoi"
    with vk.batch_from_workloads(ws, rule="voronoi", v0=0.3) as sim:
        sim.step(30)
        batch = [sim.state(r) for r in range(len(ws))]
        for r, w in enumerate(ws):
            off, ids = sim.neighbors(r)
            woff, wids = oracle.voronoi(batch[r][0], w.box_q)
            assert np.array_equal(off, woff) and np.array_equal(ids, wids)
    for r in (1, 3, 4):
        with vk.from_workload(ws[r], replica_offset=r, rule="voronoi", v0=0.3) as sim:
            sim.step(30)
            pos, d, _, _ = sim.state()
        assert np.array_equal(pos, batch[r][0]) and np.array_equal(d, batch[r][1])
