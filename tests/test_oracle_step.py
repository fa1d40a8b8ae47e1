"""Pins for the oracle's Vicsek update: Eq. (1) advection and Eq. (2)
alignment with noise (Sec. "Metric and topological flocking models").

Pins: hand-worked cases (tests/golden), the eta = 0 invariant (a flock of
equal headings stays perfectly ordered, phi = 1), the eta = 2pi limit where
headings are independent and uniform so N*phi^2 ~ Exp(1) and
E[phi] = sqrt(pi)/(2 sqrt(N)) (Rayleigh), and the advection compared with
exact rational arithmetic including half-way rounding and wrap-around.
At 0 < eta < 2pi: the angular kick's range, mean and variance (uniform on
[-eta/2, eta/2)), and for the vectorial form the bisection identity (when
|S/m| = |eta xi| the new heading is the mean angle of S/m and xi) and the
cone bound asin(eta/|S/m|), which fix the weighting by 1/m including self.
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


def _aligned_case(n, m, theta_e=0.7, include_self=False, self_opposite=False):
    """n particles that each have m neighbors, every neighbor heading along
    theta_e (so the direction of the neighbor sum is known exactly).  With
    self_opposite the particles themselves point the other way."""
    e = np.array([math.cos(theta_e), math.sin(theta_e)], dtype=np.float32)
    d = np.tile(e, (n + m, 1))
    if self_opposite:
        d[:n] = -e
    rows = [[n + j for j in range(m)] for _ in range(n)] + [[] for _ in range(m)]
    off, ids = _csr(rows)
    pos = np.zeros((n + m, 2), dtype=np.int32)
    return pos, d, off, ids, math.atan2(float(e[1]), float(e[0]))


def _wrap_pi(x):
    return (np.asarray(x) + math.pi) % (2 * math.pi) - math.pi


@pytest.mark.parametrize("eta", [1.0, 0.1])
def test_angular_noise_is_uniform_on_minus_half_eta_to_half_eta(orc, eta):
    """Reading A1 of Eq. (2): the angular kick is uniform on [-eta/2, eta/2).
    With every neighbor heading along theta_e the aligned direction is
    theta_e exactly, so theta' - theta_e is the kick itself: it must lie in
    [-eta/2, eta/2), have mean 0 (within 4 sigma, sigma = eta/sqrt(12 N)) and
    variance eta^2/12 (within 4 standard errors of a uniform variance).  A
    dropped -1/2 shifts the mean by eta/2; a kick scaled by 2pi leaves the
    range."""
    n = 20000
    pos, d, off, ids, th_e = _aligned_case(n, 3)
    eta32 = float(np.float32(eta))
    _, _, th = orc.vicsek_step(pos, d, (1 << 20, 1 << 20), off, ids, frac_bits=0, v0=0.0, dt=1.0,
                               eta=eta, seed=11, step=4)
    dev = _wrap_pi(th[:n] - th_e)
    assert dev.min() >= -eta32 / 2 - 1e-12 and dev.max() < eta32 / 2 + 1e-12
    sigma = eta32 / math.sqrt(12 * n)
    assert abs(dev.mean()) < 4 * sigma
    var_want = eta32 ** 2 / 12
    # variance of the sample variance of U(-a, a): (mu4 - sigma^4)/n, mu4 = a^4/5
    a = eta32 / 2
    se_var = math.sqrt((a ** 4 / 5 - var_want ** 2) / n)
    assert abs(dev.var() - var_want) < 4 * se_var
    # the kick spans the whole interval
    assert dev.min() < -eta32 / 2 + 20 * eta32 / n and dev.max() > eta32 / 2 - 20 * eta32 / n


@pytest.mark.parametrize("m,include_self,eta", [(2, False, 1.0), (3, False, 1.0), (3, True, 1.0 / 3.0)])
def test_vectorial_noise_half_angle_identity(orc, m, include_self, eta):
    """Eq. (2) literally, n' = N(eta xi + S/m), xi = (cos 2pi u, sin 2pi u).
    When S/m and eta*xi have equal length their sum bisects them, so the new
    heading is the mean of the two angles: theta' = (theta_e + 2 pi u)/2
    (mod pi), within pi/2 of theta_e.  Cases:
      * m = 2 or 3 aligned neighbors, eta = 1: |S/m| = 1 only if the sum is
        divided by m;
      * include_self with the particle pointing against its two aligned
        neighbors, eta = 1/3: S = e, m = 3 (self counted), |S/m| = 1/3.
    u comes from the Philox4x32-10 block of (seed, id, step, replica), pinned
    separately against PyTorch's generator."""
    n = 4000
    n_nb = m - 1 if include_self else m
    pos, d, off, ids, th_e = _aligned_case(n, n_nb, include_self=include_self, self_opposite=include_self)
    seed, step = 123456789, 17
    _, _, th = orc.vicsek_step(pos, d, (1 << 20, 1 << 20), off, ids, frac_bits=0, v0=0.0, dt=1.0,
                               eta=eta, seed=seed, step=step, noise="vectorial",
                               include_self=include_self)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    u = np.array([(int(orc.philox4x32_10((i, step, 0, 0), key)[0]) >> 8) * 2.0 ** -24
                  for i in range(n)])
    dev = _wrap_pi(th[:n] - th_e)
    want = _wrap_pi(math.pi * u - th_e / 2)
    want = np.where(want >= math.pi / 2, want - math.pi, want)
    # |e| = 1 and eta = 1/3 hold only to FP32 precision (~6e-8), so the
    # bisection holds to ~1e-7 divided by the length of the sum, 2|cos(want)|
    err = np.abs(_wrap_pi(dev - want))
    assert np.all(err < 2e-7 / np.abs(np.cos(want)) + 1e-12), err.max()
    # and the deviation is uniform on [-pi/2, pi/2)
    assert abs(dev.mean()) < 4 * math.pi / math.sqrt(12 * n)


def test_vectorial_noise_deviation_bound(orc):
    """With |S/m| = 1 and eta = 1/2 < 1 the noisy vector stays in the cone of
    half-angle asin(1/2) = pi/6 around S/m, and over many draws comes close
    to its edge.  If the sum were not divided by m (m = 3) the cone would be
    asin(1/6)."""
    n = 20000
    pos, d, off, ids, th_e = _aligned_case(n, 3)
    _, _, th = orc.vicsek_step(pos, d, (1 << 20, 1 << 20), off, ids, frac_bits=0, v0=0.0, dt=1.0,
                               eta=0.5, seed=5, step=2, noise="vectorial")
    dev = np.abs(_wrap_pi(th[:n] - th_e))
    assert dev.max() <= math.pi / 6 + 1e-12
    assert dev.max() > math.pi / 6 - 1e-3
