"""Precision study of the FP32 dynamics (a script, not collected by pytest).

The workload is the density-2 uniform flock (N = 2^20 by default, F = 20,
eta = 0.25), for the k-nearest (k = 7) and the Voronoi rule.  For each
heading-sum mode (FP32 plain, FP32 compensated, FP64) one free run of
--steps steps takes a teacher-forced check every --check-every steps:

* the neighbor lists of the checked state against the oracle (kNN: a random
  sample of 4096 particles against brute force over all N; Voronoi: every
  list against the exact Delaunay triangulation);
* one step: positions bit-exact against the oracle step from the same state
  and lists, and the heading error of every particle against the oracle's
  FP64 heading (Eq. 2 with angular noise, reading A1), with the magnitude of
  the neighbor sum |S| of the particles above 1e-5 rad (the near-cancelling
  sums that plain FP32 summation loses);
* the order parameter of every step, time-averaged over the second half of
  the run with a standard error from 20 blocks (free-running trajectories of
  different precisions separate chaotically, so they compare statistically).

Usage (on a GPU machine):  python tests/precision_study.py --out results.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)


def run(n: int, steps: int, check_every: int, rules, stream=None, seed: int = 5) -> dict:
    import oracle
    from paper_2103_10239_gb300 import vk
    from paper_2103_10239_gb300 import workloads as W
    from parity import angle_between
    oracle.build()
    rng = np.random.default_rng(seed)
    out = {}
    for rule in rules:
        w = W.precision_study(rule, n=n)
        for mode in ("plain", "compensated", "fp64"):
            t_start = time.perf_counter()
            checks = []
            with vk.from_workload(w, stream=stream, sum_mode=mode, phi_capacity=steps + 2) as sim:
                done = 0
                while done < steps:
                    n_free = min(check_every - 1, steps - done - 1)
                    if n_free > 0:
                        sim.step(n_free)
                        done += n_free
                    pos0, d0, _, t0 = sim.state()
                    off, ids = sim.neighbors()
                    if rule == "knn":
                        q = np.sort(rng.choice(w.n, min(4096, w.n), replace=False)).astype(np.int64)
                        lists_ok = bool(np.array_equal(ids.reshape(-1, w.k)[q],
                                                       oracle.knn(pos0, w.box_q, w.k, query=q)))
                    else:
                        woff, wids = oracle.voronoi(pos0, w.box_q)
                        lists_ok = bool(np.array_equal(off, woff) and np.array_equal(ids, wids))
                    sim.step(1)
                    done += 1
                    pos1, d1, _, _ = sim.state()
                    op, od, _ = oracle.vicsek_step(pos0, d0, w.box_q, off, ids, frac_bits=w.frac_bits, v0=w.v0,
                                                   dt=w.dt, eta=w.eta, seed=w.seed, step=t0)
                    err = angle_between(d1, od)
                    bad = np.nonzero(err > 1e-5)[0]
                    s_bad = []
                    for i in bad[:64]:
                        nb = ids[off[i]:off[i + 1]]
                        s_bad.append(float(np.hypot(*d0[nb].astype(np.float64).sum(0))))
                    checks.append({"step": int(t0), "lists_exact": lists_ok,
                                   "positions_exact": bool(np.array_equal(pos1, op)),
                                   "max_err": float(err.max()), "p9999_err": float(np.percentile(err, 99.99)),
                                   "n_above_1e-5": int(bad.size), "S_of_those": sorted(s_bad)[:8]})
                phi = sim.order_parameter()
            half = phi[len(phi) // 2:]
            bm = np.array([b.mean() for b in np.array_split(half, 20)])
            res = {"n": w.n, "steps": int(steps), "check_every": int(check_every),
                   "max_err_over_checks": max(c["max_err"] for c in checks),
                   "max_p9999_over_checks": max(c["p9999_err"] for c in checks),
                   "n_above_1e-5_total": sum(c["n_above_1e-5"] for c in checks),
                   "particles_checked": len(checks) * w.n,
                   "lists_exact_all": all(c["lists_exact"] for c in checks),
                   "positions_exact_all": all(c["positions_exact"] for c in checks),
                   "phi_mean_second_half": float(half.mean()),
                   "phi_stderr": float(bm.std(ddof=1) / np.sqrt(len(bm))),
                   "wall_s": time.perf_counter() - t_start, "checks": checks}
            out[f"{rule}_{mode}"] = res
            print(json.dumps({f"{rule}_{mode}": {k: v for k, v in res.items() if k != "checks"}}), flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--check-every", type=int, default=1000)
    ap.add_argument("--rules", default="knn,voronoi")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    res = run(args.n, args.steps, args.check_every, args.rules.split(","), stream=stream)
    if args.out:
        json.dump(res, open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
