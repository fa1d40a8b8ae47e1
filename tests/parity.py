"""Shared helpers of the GPU parity tests: the teacher-forced comparison of
one CUDA step with one oracle step from the same state.

Tolerances:
  * neighbor lists and positions: bit-exact (integer work);
  * headings: angle between the GPU's FP32 heading and the oracle's FP64
    heading <= 1e-5 rad per step (the bound stated for the FP32 dynamics);
  * order parameter: |dphi| <= 1e-6.
"""
import numpy as np

import oracle

HEADING_TOL = 1e-5
PHI_TOL = 1e-6


def angle_between(a, b) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.shape[1] == 2:
        cross = a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
        return np.abs(np.arctan2(cross, (a * b).sum(1)))
    c = np.cross(a, b)
    return np.arctan2(np.linalg.norm(c, axis=1), (a * b).sum(1))


def oracle_neighbors(pos, box, rule, k):
    if rule == "knn":
        return oracle.csr_from_dense(oracle.knn(pos, box, k))
    if np.asarray(pos).shape[1] == 3:
        return oracle.voronoi3(pos, box)
    return oracle.voronoi(pos, box)


def check_step(sim, w, rule, *, replica=0, check_neighbors=True, lists=None, **step_kw):
    """Compare neighbor lists of the current state, then one step.
    ``lists(pos, dir) -> (offsets, ids)`` gives the oracle's lists for rules
    other than plain kNN and Voronoi."""
    pos0, d0, _, t0 = sim.state(replica)
    if lists is not None:
        off_o, ids_o = lists(pos0, d0)
    else:
        off_o, ids_o = oracle_neighbors(pos0, w.box_q, rule, w.k)
    if check_neighbors:
        off_g, ids_g = sim.neighbors(replica)
        assert np.array_equal(off_g, off_o), "neighbor counts differ"
        assert np.array_equal(ids_g, ids_o), "neighbor ids differ"
    sim.step(1)
    pos1, d1, th1, t1 = sim.state(replica)
    assert t1 == t0 + 1
    kw = dict(frac_bits=w.frac_bits, v0=w.v0, dt=w.dt, eta=w.eta, seed=w.seed, step=t0,
              replica=replica, noise=w.noise)
    kw.update(step_kw)
    op, od, oth = oracle.vicsek_step(pos0, d0, w.box_q, off_o, ids_o, **kw)
    if not kw.get("advect_new"):
        assert np.array_equal(pos1, op), "positions differ"
    else:
        assert np.abs(pos1.astype(np.int64) - op).max() <= 1
    err = angle_between(d1, od)
    assert err.max() <= HEADING_TOL, f"heading error {err.max():.3e}"
    return pos1, d1, od, err.max()
