"""Pins for the oracle's 3D Voronoi-neighbor rule.

Sec. "Computational tools: Voronoi neighbor lists": a particle's Voronoi cell
holds the points closer to it than to any other particle, and two particles
are neighbors when their cells share a face; in 3D the dual Delaunay
triangulation has the empty-circumsphere property.  The oracle builds every
cell by exact clipping with the bisector half-spaces and keeps the sites whose
plane carries a face of positive area.  Pins, none of which reuses the
oracle's arithmetic:
  * lattices with closed-form neighbor counts, whose cells are degenerate
    (simple cubic: 6 of the 26 shell sites, the cube; body-centred cubic: 14,
    the truncated octahedron; face-centred cubic: 12, the rhombic
    dodecahedron, whose second shell touches only at vertices; orthorhombic
    with three distinct edges: 6);
  * the cells tile the box: their volumes add up to the box volume;
  * reciprocity of the lists;
  * scipy's Qhull Delaunay triangulation on generic tiled inputs;
  * the exact vertex test against exact rational arithmetic.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

from paper_2103_10239_gb300 import workloads as W


def _rows(off, ids):
    return [list(map(int, ids[off[i]:off[i + 1]])) for i in range(off.shape[0] - 1)]


def _lattice_shell(pos, box, i, shell_offsets):
    """ids of the particles at the given offsets (exact, periodic) from i"""
    where = {tuple(p): t for t, p in enumerate(pos.tolist())}
    out = []
    for o in shell_offsets:
        q = tuple(int((pos[i][a] + o[a]) % box[a]) for a in range(3))
        out.append(where[q])
    return sorted(out)


@pytest.mark.parametrize("m,a,off", [(4, 64, (0, 0, 0)), (5, 6, (3, 1, 2)), (3, 1000, (999, 0, 500))])
def test_simple_cubic_has_the_six_face_neighbors(orc, m, a, off):
    """Eight cubes meet at every vertex and four at every edge: only the six
    face-sharing sites count."""
    pos, box = W.cubic_lattice("sc", m, a, off)
    off_, ids = orc.voronoi3(pos, box)
    rows = _rows(off_, ids)
    six = [(a, 0, 0), (-a, 0, 0), (0, a, 0), (0, -a, 0), (0, 0, a), (0, 0, -a)]
    for i in range(pos.shape[0]):
        assert rows[i] == _lattice_shell(pos, box, i, six)


def test_body_centred_cubic_has_fourteen(orc):
    pos, box = W.cubic_lattice("bcc", 4, 64, (5, 7, 9))
    off, ids = orc.voronoi3(pos, box)
    rows = _rows(off, ids)
    h = 32
    shell = [(sx * h, sy * h, sz * h) for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]
    shell += [(64, 0, 0), (-64, 0, 0), (0, 64, 0), (0, -64, 0), (0, 0, 64), (0, 0, -64)]
    for i in range(pos.shape[0]):
        assert rows[i] == _lattice_shell(pos, box, i, shell)


def test_face_centred_cubic_has_twelve(orc):
    """The second shell (+-a, 0, 0) meets the rhombic dodecahedron in a
    vertex only, where six cells meet: it must not count."""
    pos, box = W.cubic_lattice("fcc", 4, 64)
    off, ids = orc.voronoi3(pos, box)
    rows = _rows(off, ids)
    shell = [p for p in itertools.product((-32, 0, 32), repeat=3) if sorted(map(abs, p)) == [0, 32, 32]]
    assert len(shell) == 12
    for i in range(pos.shape[0]):
        assert rows[i] == _lattice_shell(pos, box, i, shell)


def test_orthorhombic_lattice_has_six(orc):
    """Three distinct edges a < b < c: the cell is a box, 6 faces."""
    pos, box = W.cubic_lattice("sc", (5, 4, 3), (30, 41, 57))
    off, ids = orc.voronoi3(pos, box)
    assert set(np.diff(off).tolist()) == {6}


def test_centred_lattices_in_stretched_boxes(orc):
    """A body-centred orthorhombic lattice with a < b < c and c^2 < a^2 + b^2
    gives the truncated octahedron again (14): the 8 centres and the 6
    corner sites along the three edges."""
    pos, box = W.cubic_lattice("bcc", (4, 4, 4), (40, 44, 48))
    off, ids = orc.voronoi3(pos, box)
    assert set(np.diff(off).tolist()) == {14}
    off, ids, vol = orc.voronoi3(pos, box, volumes=True)
    assert np.allclose(vol, box[0] * box[1] * box[2] / pos.shape[0], rtol=1e-12)


@pytest.mark.parametrize("n,L,seed", [(500, 1 << 14, 1), (3000, 1 << 20, 2), (40, 100, 3)])
def test_cells_tile_the_box(orc, n, L, seed):
    """Volumes of all cells add up to the box volume, each cell has positive
    volume, and the neighbor relation is reciprocal."""
    rng = np.random.default_rng(seed)
    pos = rng.integers(0, L, size=(n, 3)).astype(np.int32)
    if len({tuple(p) for p in pos.tolist()}) < n:
        pytest.skip("coincident draw")
    off, ids, vol = orc.voronoi3(pos, (L, L, L), volumes=True)
    assert (vol > 0).all()
    assert abs(vol.sum() / float(L) ** 3 - 1.0) < 1e-11
    pairs = {(i, int(j)) for i in range(n) for j in ids[off[i]:off[i + 1]]}
    assert all((j, i) in pairs for (i, j) in pairs)


@pytest.mark.parametrize("box,n,seed", [((1000, 1700, 2900), 300, 4), ((64, 64, 640), 50, 5),
                                        ((37, 41, 43), 3, 6), ((100, 100, 100), 2, 7),
                                        ((20, 200, 20), 4, 8)])
def test_stretched_and_tiny_boxes_tile(orc, box, n, seed):
    """Small and elongated boxes: a cell meets several periodic images of a
    particle, including its own; the volumes still add up to the box."""
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.integers(0, b, size=n) for b in box], axis=1).astype(np.int32)
    if len({tuple(p) for p in pos.tolist()}) < n:
        pytest.skip("coincident draw")
    off, ids, vol = orc.voronoi3(pos, box, volumes=True)
    assert (vol > 0).all()
    assert abs(vol.sum() / float(np.prod(box)) - 1.0) < 1e-11
    for i in range(n):
        assert i not in set(ids[off[i]:off[i + 1]].tolist())


def test_single_particle_and_pair(orc):
    off, ids = orc.voronoi3(np.array([[5, 6, 7]], dtype=np.int32), (50, 60, 70))
    assert off.tolist() == [0, 0]
    off, ids, vol = orc.voronoi3(np.array([[5, 6, 7], [30, 20, 51]], dtype=np.int32), (50, 60, 70),
                                 volumes=True)
    assert _rows(off, ids) == [[1], [0]]
    assert np.allclose(vol, [50 * 60 * 70 / 2] * 2, rtol=1e-12)


def _qhull_rows(pos, box, reach):
    spatial = pytest.importorskip("scipy.spatial")
    n = pos.shape[0]
    shifts = list(itertools.product(range(-reach, reach + 1), repeat=3))
    pts = np.concatenate([pos.astype(np.float64) + np.array(s) * np.array(box, dtype=np.float64)
                          for s in shifts])
    owner = np.tile(np.arange(n), len(shifts))
    c0 = shifts.index((0, 0, 0)) * n
    tri = spatial.Delaunay(pts)
    want = [set() for _ in range(n)]
    for simplex in tri.simplices:
        for a in simplex:
            if c0 <= a < c0 + n:
                for b in simplex:
                    if owner[b] != owner[a]:
                        want[a - c0].add(int(owner[b]))
    return [sorted(s) for s in want]


def test_against_qhull_on_generic_input(orc):
    w = W.uniform_system(400, 400 ** (1 / 3), 16, 3, input_seed=31)
    off, ids = orc.voronoi3(w.pos_q, w.box_q)
    assert _rows(off, ids) == _qhull_rows(w.pos_q, w.box_q, 1)


def test_against_qhull_on_jittered_lattice(orc):
    """A body-centred lattice jittered by a few grid units: nearly degenerate
    (nearly cospherical groups), still generic."""
    pos, box = W.cubic_lattice("bcc", 3, 4000)
    rng = np.random.default_rng(9)
    pos = np.mod(pos + rng.integers(-60, 61, size=pos.shape), np.array(box)).astype(np.int32)
    off, ids, vol = orc.voronoi3(pos, box, volumes=True)
    assert _rows(off, ids) == _qhull_rows(pos, box, 1)
    assert abs(vol.sum() / float(np.prod(box)) - 1.0) < 1e-11


def test_against_qhull_in_a_tiny_box(orc):
    """Five particles: the cells reach several images of every particle."""
    rng = np.random.default_rng(12)
    box = (3000, 3500, 4100)
    pos = np.stack([rng.integers(0, b, size=5) for b in box], axis=1).astype(np.int32)
    off, ids = orc.voronoi3(pos, box)
    assert _rows(off, ids) == _qhull_rows(pos, box, 2)


def test_query_rows_match_the_full_run(orc):
    w = W.uniform_system(1500, 1500 ** (1 / 3), 18, 3, input_seed=33)
    off, ids = orc.voronoi3(w.pos_q, w.box_q)
    q = np.array([0, 7, 1499, 700, 7])
    offq, idsq = orc.voronoi3(w.pos_q, w.box_q, query=q)
    rows = _rows(off, ids)
    assert _rows(offq, idsq) == [rows[i] for i in q]


def test_coincident_particles_are_degenerate(orc):
    pos = np.array([[1, 2, 3], [400, 500, 600], [1, 2, 3]], dtype=np.int32)
    with pytest.raises(orc.OracleError):
        orc.voronoi3(pos, (1000, 1000, 1000))


def test_box_range(orc):
    pos = np.array([[1, 2, 3], [400, 500, 600]], dtype=np.int32)
    with pytest.raises(orc.OracleError):
        orc.voronoi3(pos, (1 << 29, 1000, 1000))


def _side_rational(da, db, dc, de):
    """sign(d_e.y - |d_e|^2) with y solving d_x.y = |d_x|^2 (x = a, b, c), by
    Gaussian elimination over the rationals"""
    rows = [[Fraction(v) for v in d] + [Fraction(sum(t * t for t in d))] for d in (da, db, dc)]
    for c in range(3):
        p = next(r for r in range(c, 3) if rows[r][c] != 0)
        rows[c], rows[p] = rows[p], rows[c]
        for r in range(3):
            if r != c and rows[r][c] != 0:
                f = rows[r][c] / rows[c][c]
                rows[r] = [x - f * y for x, y in zip(rows[r], rows[c])]
    y = [rows[c][3] / rows[c][c] for c in range(3)]
    v = sum(Fraction(e) * t for e, t in zip(de, y)) - sum(t * t for t in de)
    return (v > 0) - (v < 0)


def test_exact_vertex_test_against_rationals(orc):
    rng = np.random.default_rng(13)
    checked = 0
    for scale in (10, 1 << 12, 1 << 22, 1 << 27):
        for _ in range(300):
            d = rng.integers(-scale, scale + 1, size=(4, 3))
            if round(np.linalg.det(d[:3].astype(np.float64))) == 0:
                continue
            if len({tuple(r) for r in d.tolist()}) < 4:
                continue
            da, db, dc, de = (list(map(int, r)) for r in d)
            assert orc.voronoi3_side(da, db, dc, de) == _side_rational(da, db, dc, de)
            checked += 1
    # exactly on the plane: the cube corner (1,1,1)*a of planes 2a e_x, 2a e_y, 2a e_z
    # lies on the planes of (2a, 2a, 0) and (2a, 2a, 2a); (2a, 2a, a) cuts it
    for a in (1, 1000, 1 << 26):
        ax, ay, az = [2 * a, 0, 0], [0, 2 * a, 0], [0, 0, 2 * a]
        assert orc.voronoi3_side(ax, ay, az, [2 * a, 2 * a, 0]) == 0
        assert orc.voronoi3_side(ax, ay, az, [2 * a, 2 * a, 2 * a]) == 0
        assert orc.voronoi3_side(ax, ay, az, [2 * a, 2 * a, a]) == 1
        assert orc.voronoi3_side(ax, ay, az, [2 * a, 2 * a, 3 * a]) == -1
    assert checked > 1000
