"""Pins for the oracle's Vicsek update: Eq. (1) advection and Eq. (2)
alignment with noise (Sec. "Metric and topological flocking models").

Pins: hand-worked cases (tests/golden), the eta = 0 invariant (a flock of
equal headings stays perfectly ordered, phi = 1), the eta = 2pi limit where
headings are independent and uniform so N*phi^2 ~ Exp(1) and
E[phi] = sqrt(pi)/(2 sqrt(N)) (Rayleigh), and the advection compared with
exact rational arithmetic including half-way rounding and wrap-around.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2103_10239_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "align_advect_hand_worked.json")


def _csr(rows):
    off = np.zeros(len(rows) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    ids = np.array([j for r in rows for j in r], dtype=np.int32)
    return off, ids


def test_hand_worked_alignment(orc):
    g = json.load(open(GOLD))
    for case in g["alignment"]:
        d = np.array(case["dir"], dtype=np.float32)
        n = d.shape[0]
        off, ids = _csr(case["neighbors"])
        pos = np.zeros((n, 2), dtype=np.int32)
        for noise in ("angular", "vectorial"):
            _, dout, th = orc.vicsek_step(pos, d, (1000, 1000), off, ids, frac_bits=0, v0=0.0,
                                          dt=1.0, eta=0.0, seed=1, step=0, noise=noise,
                                          include_self=case.get("include_self", False))
            want = np.array(case["expected_theta_over_pi"]) * math.pi
            assert np.allclose(th, want, atol=1e-14), (case["citation"], noise, th, want)
            assert np.allclose(dout, np.stack([np.cos(want), np.sin(want)], 1), atol=1e-14)


def test_hand_worked_advection(orc):
    g = json.load(open(GOLD))["advection"]
    for c in g["cases"]:
        pos = np.array([c["pos"]], dtype=np.int32)
        d = np.array([c["dir"]], dtype=np.float32)
        off, ids = _csr([[]])
        pout, _, _ = orc.vicsek_step(pos, d, g["box_q"], off, ids, frac_bits=g["frac_bits"],
                                     v0=g["v0"], dt=g["dt"], eta=0.0, seed=1, step=0)
        assert list(pout[0]) == c["expected"], c


def test_advection_exact_against_rationals(orc):
    rng = np.random.default_rng(5)
    n = 3000
    for F, L, v0, dt in [(16, 2965504, 0.5, 1.0), (20, 1 << 31, 0.5, 1.0), (16, 12345, 0.3, 0.7),
                         (20, 759250125, 0.123, 2.0)]:
        pos = rng.integers(0, L, size=(n, 2)).astype(np.int32)
        pos[:10] = 0
        pos[10:20] = L - 1
        d = W.random_dirs(n, 2, seed=F)
        # include exact half-way products
        d[20] = np.float32(2.0 ** -F) * np.array([1, 3], dtype=np.float32) / np.float32(v0 * dt) \
            if v0 * dt == 0.5 else d[20]
        off, ids = _csr([[] for _ in range(n)])
        pout, _, _ = orc.vicsek_step(pos, d, (L, L), off, ids, frac_bits=F, v0=v0, dt=dt,
                                     eta=0.0, seed=1, step=0)
        s = Fraction(float(np.float32(np.float32(v0) * np.float32(dt)))) * (1 << F)
        for i in range(0, n, 7):
            for a in range(2):
                delta = round(s * Fraction(float(d[i, a])))  # round-half-even on Fractions
                assert int(pout[i, a]) == (int(pos[i, a]) + delta) % L


def test_zero_noise_keeps_an_ordered_flock(orc):
    w = W.uniform_system(1500, 38.0, 16, 2, input_seed=3)
    ang = np.float32(1.234)
    d = np.tile(np.array([np.cos(ang), np.sin(ang)], dtype=np.float32), (w.n, 1))
    off, ids = orc.neighbors(w.pos_q, w.box_q, "knn", 7)
    _, dout, _ = orc.vicsek_step(w.pos_q, d, w.box_q, off, ids, frac_bits=16, v0=0.5, dt=1.0,
                                 eta=0.0, seed=1, step=0)
    assert abs(orc.order_parameter(dout) - 1.0) < 1e-12
    want = math.atan2(float(d[0, 1]), float(d[0, 0]))
    assert np.allclose(np.arctan2(dout[:, 1], dout[:, 0]), want, atol=1e-14)


def test_full_noise_gives_rayleigh_statistics(orc):
    """eta = 2pi: theta' = theta* + 2pi(u - 1/2) is uniform on the circle for
    any theta*, so N phi^2 is Exp(1) and E[phi] = sqrt(pi)/(2 sqrt(N))."""
    w = W.topological_small()
    off, ids = orc.neighbors(w.pos_q, w.box_q, "knn", 7)
    vals = []
    for t in range(300):
        _, dout, _ = orc.vicsek_step(w.pos_q, w.dir, w.box_q, off, ids, frac_bits=16, v0=0.5,
                                     dt=1.0, eta=2 * math.pi, seed=1, step=t)
        vals.append(orc.order_parameter(dout))
    vals = np.array(vals)
    nphi2 = w.n * vals ** 2
    assert abs(nphi2.mean() - 1.0) < 4 / math.sqrt(len(vals))
    want = math.sqrt(math.pi) / (2 * math.sqrt(w.n))  # 0.01958 at N = 2048
    assert abs(vals.mean() - want) < 4 * want * math.sqrt(4 / math.pi - 1) / math.sqrt(len(vals))


def test_vectorial_noise_3d_direction_is_uniform(orc):
    """With no neighbors (S = 0) and eta = 1 the vectorial rule returns xi,
    which must be uniform on the sphere: mean ~ 0 and <z^2> = 1/3."""
    n = 20000
    pos = np.zeros((n, 3), dtype=np.int32)
    d = W.random_dirs(n, 3, seed=4)
    off = np.zeros(n + 1, dtype=np.int64)
    _, dout, _ = orc.vicsek_step(pos, d, (100, 100, 100), off, np.zeros(0, np.int32), frac_bits=0,
                                 v0=0.0, dt=1.0, eta=1.0, seed=9, step=3, noise="vectorial")
    assert np.allclose(np.linalg.norm(dout, axis=1), 1.0, atol=1e-12)
    assert np.all(np.abs(dout.mean(0)) < 4 / math.sqrt(3 * n))
    assert abs((dout[:, 2] ** 2).mean() - 1 / 3) < 4 * math.sqrt(4 / 45 / n)


def test_noise_is_keyed_by_id_step_replica(orc):
    """Counter-based noise: the same (seed, id, step, replica) always gives
    the same draw; changing any of them changes it."""
    w = W.uniform_system(64, 8.0, 16, 2, input_seed=2)
    off, ids = orc.neighbors(w.pos_q, w.box_q, "knn", 7)
    kw = dict(frac_bits=16, v0=0.5, dt=1.0, eta=1.0)
    a = orc.vicsek_step(w.pos_q, w.dir, w.box_q, off, ids, seed=1, step=5, **kw)[1]
    b = orc.vicsek_step(w.pos_q, w.dir, w.box_q, off, ids, seed=1, step=5, **kw)[1]
    assert np.array_equal(a, b)
    for other in [dict(seed=2, step=5), dict(seed=1, step=6), dict(seed=1, step=5, replica=1)]:
        c = orc.vicsek_step(w.pos_q, w.dir, w.box_q, off, ids, **other, **kw)[1]
        assert not np.allclose(a, c)


def test_order_parameter_definition(orc):
    d = np.array([[1, 0], [0, 1], [-1, 0], [0, 1]], dtype=np.float32)
    assert abs(orc.order_parameter(d) - 0.5) < 1e-15  # |(0, 2)| / 4
