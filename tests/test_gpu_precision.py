"""Precision study (FP32 plain vs FP32 compensated vs FP64 heading sums) on
the density-2 uniform workload (N = 2^20), both rules, after the flock has evolved:
per-step heading error against the FP64 oracle with teacher forcing, and the
neighbor lists bit-exact.  Compensated sums and FP64 must stay within
1e-5 rad per step; plain FP32 sums are reported (they can exceed it when the
neighbor headings nearly cancel)."""
import numpy as np
import pytest

import oracle
from paper_2103_10239_gb300 import vk
from paper_2103_10239_gb300 import workloads as W
from parity import angle_between

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rule", ["voronoi", "knn"])
def test_heading_error_by_sum_mode(rule):
    """At the study's size (N = 2^20, density 2): one teacher-forced check
    after 30 free steps.  The long runs (10^4 steps, a check every 1000) are
    tests/precision_study.py."""
    w = W.precision_study(rule, n=1 << 20)
    rng = np.random.default_rng(3)
    report = {}
    for mode in ("plain", "compensated", "fp64"):
        with vk.from_workload(w, sum_mode=mode) as sim:
            sim.step(30)
            pos0, d0, _, t0 = sim.state()
            off, ids = sim.neighbors()
            if rule == "knn":
                q = np.sort(rng.choice(w.n, 2048, replace=False))
                assert np.array_equal(ids.reshape(-1, 7)[q], oracle.knn(pos0, w.box_q, 7, query=q))
            else:
                woff, wids = oracle.voronoi(pos0, w.box_q)
                assert np.array_equal(off, woff) and np.array_equal(ids, wids)
                q = np.arange(w.n)
            sim.step(1)
            pos1, d1, _, _ = sim.state()
            op, od, _ = oracle.vicsek_step(pos0, d0, w.box_q, off, ids, frac_bits=w.frac_bits, v0=w.v0,
                                           dt=w.dt, eta=w.eta, seed=w.seed, step=t0)
            assert np.array_equal(pos1[q], op[q])
            err = angle_between(d1[q], od[q])
            report[mode] = (float(err.max()), float(np.percentile(err, 99.99)), int((err > 1e-5).sum()))
    print(f"\nprecision {rule} N={w.n}: " + ", ".join(f"{m}: max {v[0]:.2e} p99.99 {v[1]:.2e} >1e-5: {v[2]}"
                                                    for m, v in report.items()))
    assert report["compensated"][0] <= 1e-5
    assert report["fp64"][0] <= 1e-5
