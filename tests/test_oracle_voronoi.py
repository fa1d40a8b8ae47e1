"""Pins for the oracle's Voronoi-neighbor rule.

Sec. "Computational tools: Voronoi neighbor lists": the Delaunay triangulation
has the empty-circumcircle property and is dual to the Voronoi diagram.  The
oracle builds the Delaunay triangulation by incremental insertion with exact
predicates and keeps an edge iff its dual Voronoi edge has positive length.
Pins: a direct bisector-clipping brute force (a different algorithm), the
empty-circumcircle property checked exhaustively, Euler's relation for a
periodic triangulation (E = 3N), lattices with known neighbor counts,
reciprocity, and scipy's Qhull triangulation on generic inputs.
"""
import numpy as np
import pytest

from oracle import brute
from paper_2103_10239_gb300 import workloads as W


def _rows(off, ids):
    return [list(map(int, ids[off[i]:off[i + 1]])) for i in range(off.shape[0] - 1)]


@pytest.mark.parametrize("seed,n,L", [(1, 12, 1 << 12), (2, 20, 3000), (3, 30, 1 << 14),
                                      (4, 5, 1 << 10), (5, 3, 999), (6, 16, 64)])
def test_voronoi_matches_bisector_brute_force(orc, seed, n, L):
    rng = np.random.default_rng(seed)
    pos = rng.integers(0, L, size=(n, 2)).astype(np.int32)
    if len({tuple(p) for p in pos}) < n:
        pytest.skip("coincident draw")
    off, ids = orc.voronoi(pos, (L, L))
    assert _rows(off, ids) == brute.voronoi_brute(pos, (L, L))


def test_voronoi_brute_force_on_degenerate_lattices(orc):
    pos, box = W.square_lattice(5, 40)
    off, ids = orc.voronoi(pos, box)
    assert _rows(off, ids) == brute.voronoi_brute(pos, box)
    pos, box = W.stretched_hex_lattice(4, 6, 40, 35)
    off, ids = orc.voronoi(pos, box)
    assert _rows(off, ids) == brute.voronoi_brute(pos, box)


@pytest.mark.parametrize("n,seed", [(200, 1), (2000, 2)])
def test_euler_relation_generic(orc, n, seed):
    """Periodic triangulation of N generic points: V - E + F = 0 and
    3F = 2E give E = 3N, so the directed neighbor count is 6N."""
    w = W.uniform_system(n, np.sqrt(n), 16, 2, input_seed=seed)
    off, ids = orc.voronoi(w.pos_q, w.box_q)
    assert ids.size == 6 * n


def test_square_lattice_has_four_neighbors(orc):
    """Cocircular squares: the diagonal's Voronoi edge has zero length."""
    for m, a, o in [(8, 1 << 16, 0), (5, 7, 3), (12, 1000, 999)]:
        pos, box = W.square_lattice(m, a, o)
        off, ids = orc.voronoi(pos, box)
        assert set(np.diff(off)) == {4}
        assert ids.size == 4 * pos.shape[0]  # E = 2N undirected edges


def test_hex_lattice_has_six_neighbors(orc):
    pos, box = W.stretched_hex_lattice(16, 18, 2 * 1000, 866)
    off, ids = orc.voronoi(pos, box)
    assert set(np.diff(off)) == {6}


def test_reciprocity_on_workload_shape(orc):
    w = W.voronoi_mixed()
    sub = w.pos_q  # full 65536 configuration
    off, ids = orc.voronoi(sub, w.box_q)
    rows = _rows(off, ids)
    sets = [set(r) for r in rows]
    for i, r in enumerate(rows):
        for j in r:
            assert i in sets[j]
    # mixed uniform/lattice input is generic after jitter: E = 3N
    assert ids.size == 6 * w.n


def test_empty_circumcircle_exhaustive(orc):
    """Every triangle around an original point has no site strictly inside
    its circumcircle (checked against all 5x5 periodic images)."""
    rng = np.random.default_rng(9)
    L = 1 << 12
    for trial in range(4):
        n = int(rng.integers(4, 40))
        pos = rng.integers(0, L, size=(n, 2)).astype(np.int32)
        coords, tids = orc.delaunay_star_triangles(pos, (L, L))
        sx, sy = np.meshgrid(np.arange(-2, 3), np.arange(-2, 3))
        sites = (pos[None, :, :].astype(np.int64)
                 + np.stack([sx.ravel(), sy.ravel()], 1)[:, None, :] * L).reshape(-1, 2)
        for t in range(coords.shape[0]):
            a, b, c = coords[t]
            assert brute.orient_int(a, b, c) > 0
            d = sites - c
            adx, ady = a[0] - sites[:, 0], a[1] - sites[:, 1]
            bdx, bdy = b[0] - sites[:, 0], b[1] - sites[:, 1]
            cdx, cdy = c[0] - sites[:, 0], c[1] - sites[:, 1]
            det = ((adx * adx + ady * ady) * (bdx * cdy - bdy * cdx)
                   + (bdx * bdx + bdy * bdy) * (cdx * ady - cdy * adx)
                   + (cdx * cdx + cdy * cdy) * (adx * bdy - ady * bdx))
            # |coords| < 2^15 here, so int64 is exact
            assert (det <= 0).all()


def test_against_qhull_on_generic_input(orc):
    spatial = pytest.importorskip("scipy.spatial")
    w = W.uniform_system(600, 24.0, 16, 2, input_seed=21)
    L = w.box_q[0]
    shifts = [(sx, sy) for sy in (-1, 0, 1) for sx in (-1, 0, 1)]
    pts = np.concatenate([w.pos_q.astype(np.float64) + np.array(s) * L for s in shifts])
    owner = np.tile(np.arange(w.n), len(shifts))
    center = np.arange(w.n) + 4 * w.n  # the (0,0) copy
    tri = spatial.Delaunay(pts)
    want = [set() for _ in range(w.n)]
    for simplex in tri.simplices:
        for a in simplex:
            if 4 * w.n <= a < 5 * w.n:
                for b in simplex:
                    if b != a:
                        want[a - 4 * w.n].add(int(owner[b]))
    off, ids = orc.voronoi(w.pos_q, w.box_q)
    assert _rows(off, ids) == [sorted(s) for s in want]
    del center


def test_coincident_points_share_a_site(orc):
    """Coincident particles (reading: one Voronoi site) are each other's
    neighbors and share the site's neighbors; checked against the bisector
    brute force, which handles coincident sites without any triangulation."""
    pos = np.array([[10, 10], [500, 400], [10, 10], [900, 30], [700, 800], [10, 10], [500, 400]],
                   dtype=np.int32)
    off, ids = orc.voronoi(pos, (1000, 1000))
    rows = _rows(off, ids)
    assert rows == brute.voronoi_brute(pos, (1000, 1000))
    assert {2, 5} <= set(rows[0]) and {0, 2} <= set(rows[5]) and 6 in rows[1]
    rng = np.random.default_rng(3)
    for _ in range(30):
        n = int(rng.integers(2, 25))
        L = int(rng.integers(20, 3000))
        base = rng.integers(0, L, size=(max(1, n // 2), 2))
        pos = base[rng.integers(0, base.shape[0], size=n)].astype(np.int32)
        off, ids = orc.voronoi(pos, (L, L))
        assert _rows(off, ids) == brute.voronoi_brute(pos, (L, L))


def test_predicates(orc):
    big = 1 << 33
    assert orc.orient2d((0, 0), (big, 0), (0, big)) == 1
    assert orc.orient2d((0, 0), (0, big), (big, 0)) == -1
    assert orc.orient2d((0, 0), (big, big), (2 * big, 2 * big)) == 0
    # unit square corners are cocircular; the center is inside
    a, b, c = (0, 0), (big, 0), (big, big)
    assert orc.incircle(a, b, c, (0, big)) == 0
    assert orc.incircle(a, b, c, (big // 2, big // 2)) == 1
    assert orc.incircle(a, b, c, (-1, big)) == -1
    for _ in range(200):
        rng = np.random.default_rng(_)
        pts = [tuple(int(v) for v in rng.integers(-big, big, 2)) for _ in range(4)]
        assert orc.incircle(*pts) == brute.incircle_int(*pts)
        assert orc.orient2d(*pts[:3]) == brute.orient_int(*pts[:3])


def test_tiny_systems_against_brute_force(orc):
    """N = 1..5 in small boxes: stars whose circumdisks reach far outside the
    box (up to sqrt(2) L) -- the regime where a 3x3 tiling is not enough."""
    rng = np.random.default_rng(0)
    done = 0
    while done < 120:
        n = int(rng.integers(1, 6))
        L = int(rng.integers(8, 400))
        pos = rng.integers(0, L, size=(n, 2)).astype(np.int32)
        if len({tuple(p) for p in pos}) < n:
            continue
        off, ids = orc.voronoi(pos, (L, L))
        assert _rows(off, ids) == brute.voronoi_brute(pos, (L, L)), (n, L, pos.tolist())
        done += 1
