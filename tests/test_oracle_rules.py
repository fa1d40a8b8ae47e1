"""Pins for the oracle's metric rule and field-of-view kNN rule (Sec.
"Metric and topological flocking models": all pairs within a distance r0;
the k nearest neighbors within an angular field of view).

Pins: an independent pure-Python brute force of the metric rule; square
lattice shells (4 neighbors at r0 = a, 8 at r0 = ceil(a sqrt 2), none below
a, all at a radius beyond the box diagonal); reciprocity of the metric rule;
a full field of view reproduces the plain kNN oracle; a half-plane field of
view on a lattice keeps exactly the shells ahead; a zero-width field of view
keeps only the particles straight ahead; and random systems against an
angle-based view test in high precision (away from the cone's edge, where a
rounding of the heading may legitimately decide either way)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2103_10239_gb300 import workloads as W


def _brute_metric(pos, box, r0q):
    n = len(pos)
    rows = []
    for i in range(n):
        row = []
        for j in range(n):
            if j == i:
                continue
            D = 0
            for a in range(2):
                d = int(pos[j][a]) - int(pos[i][a])
                L = int(box[a])
                d %= L
                if 2 * d > L:
                    d -= L
                D += d * d
            if D <= r0q * r0q:
                row.append(j)
        rows.append(row)
    return rows


def test_metric_matches_python_brute_force(orc):
    rng = np.random.default_rng(2)
    for trial in range(6):
        n = int(rng.integers(2, 60))
        box = (int(rng.integers(50, 400)), int(rng.integers(50, 400)))
        pos = np.stack([rng.integers(0, box[0], n), rng.integers(0, box[1], n)], 1).astype(np.int32)
        # radii exactly at some pair distance (boundary ties) and in between
        for r0q in (0, 7, 30, int(rng.integers(1, 200))):
            off, ids = orc.metric(pos, box, r0q)
            want = _brute_metric(pos, box, r0q)
            got = [list(ids[off[i]:off[i + 1]]) for i in range(n)]
            assert got == want, (trial, r0q)


def test_metric_square_lattice_shells(orc):
    a, m = 1000, 8
    pos, box = W.square_lattice(m, a)
    for r0q, deg in ((a - 1, 0), (a, 4), (math.ceil(a * math.sqrt(2)), 8), (2 * a - 1, 8), (2 * a, 12)):
        off, ids = orc.metric(pos, box, r0q)
        assert np.all(np.diff(off) == deg), (r0q, np.unique(np.diff(off)))
    off, ids = orc.metric(pos, box, 10 ** 5)
    assert np.all(np.diff(off) == m * m - 1)


def test_metric_is_reciprocal(orc):
    w = W.uniform_system(400, 20.0, 16, 2, input_seed=5)
    off, ids = orc.metric(w.pos_q, w.box_q, int(1.3 * 2 ** 16))
    pairs = {(i, int(j)) for i in range(w.n) for j in ids[off[i]:off[i + 1]]}
    assert all((j, i) in pairs for i, j in pairs)


def test_full_field_of_view_is_plain_knn(orc):
    w = W.uniform_system(700, 26.0, 16, 2, input_seed=6)
    got, cnt = orc.knn_fov(w.pos_q, w.dir, w.box_q, 7, -1.0)
    assert np.all(cnt == 7)
    assert np.array_equal(got, orc.knn(w.pos_q, w.box_q, 7))


def test_half_plane_on_a_lattice(orc):
    """Heading exactly +x and a half-angle of 90 degrees (c = 0): a particle
    sees the half-plane dx >= 0.  On a square lattice the shells ahead are 3
    at distance a ((a,0), (0,+a), (0,-a)), 2 at a sqrt 2 ((a,+a), (a,-a)) and
    3 at 2a."""
    a, m = 1000, 9
    pos, box = W.square_lattice(m, a)
    n = m * m
    d = np.tile(np.array([[1.0, 0.0]], dtype=np.float32), (n, 1))
    for k, shell_d2 in ((3, {a * a}), (5, {a * a, 2 * a * a})):
        got, cnt = orc.knn_fov(pos, d, box, k, 0.0)
        assert np.all(cnt == k)
        for i in range(n):
            for j in got[i]:
                dx = (int(pos[j, 0]) - int(pos[i, 0])) % box[0]
                dx = dx - box[0] if 2 * dx > box[0] else dx
                dy = (int(pos[j, 1]) - int(pos[i, 1])) % box[1]
                dy = dy - box[1] if 2 * dy > box[1] else dy
                assert dx >= 0 and dx * dx + dy * dy in shell_d2


def test_zero_width_view_sees_straight_ahead_only(orc):
    a, m = 1000, 9
    pos, box = W.square_lattice(m, a)
    n = m * m
    d = np.tile(np.array([[1.0, 0.0]], dtype=np.float32), (n, 1))
    got, cnt = orc.knn_fov(pos, d, box, 3, 1.0)
    assert np.all(cnt == 3)  # (a,0), (2a,0), (3a,0) ... on the periodic row
    for i in range(n):
        for r, j in enumerate(got[i]):
            assert pos[j, 1] == pos[i, 1]
            assert (int(pos[j, 0]) - int(pos[i, 0])) % box[0] == (r + 1) * a


def test_field_of_view_against_exact_angles(orc):
    """Random systems and headings: the set of particles in view, compared
    with the angle test in exact rational arithmetic on the unrounded
    heading (cos of the angle between d and n against c, squared), for every
    pair whose cosine is not within 1e-6 of c."""
    rng = np.random.default_rng(9)
    for trial in range(4):
        n = 120
        box = (1 << 16, 1 << 16)
        pos = np.stack([rng.integers(0, box[0], n), rng.integers(0, box[1], n)], 1).astype(np.int32)
        th = rng.uniform(0, 2 * math.pi, n)
        d = np.stack([np.cos(th), np.sin(th)], 1).astype(np.float32)
        c = float(np.float32(rng.uniform(-0.9, 0.9)))
        got, cnt = orc.knn_fov(pos, d, box, n - 1, c)
        for i in range(n):
            seen = set(int(j) for j in got[i][: cnt[i]])
            nx, ny = Fraction(float(d[i, 0])), Fraction(float(d[i, 1]))
            for j in range(n):
                if j == i:
                    continue
                dx = (int(pos[j, 0]) - int(pos[i, 0])) % box[0]
                dx = dx - box[0] if 2 * dx > box[0] else dx
                dy = (int(pos[j, 1]) - int(pos[i, 1])) % box[1]
                dy = dy - box[1] if 2 * dy > box[1] else dy
                dot = dx * nx + dy * ny
                norm2 = (dx * dx + dy * dy) * (nx * nx + ny * ny)
                cos2 = dot * dot / norm2
                cosv = math.copysign(math.sqrt(float(cos2)), float(dot))
                if abs(cosv - c) < 1e-6:
                    continue
                assert (j in seen) == (cosv >= c), (trial, i, j, cosv, c)
