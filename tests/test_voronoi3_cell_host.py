"""The 3D Voronoi cell builder of the CUDA path (vk_voronoi3.cuh, plain C++
for the host and the device) compiled for the host and compared list by
list with the oracle (Sec. "Computational tools: Voronoi neighbor lists":
neighbors share a face of positive area).  The builder's exact signs and its
handling of degenerate vertices do not depend on the order in which sites
are clipped, so every case runs in index, distance and pseudo-random order.
CPU only; the device build of the same code is compared on the GPU by
test_gpu_voronoi3.py."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2103_10239_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("v3host") / "libv3host.so")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out,
                           os.path.join(HERE, "voronoi3_cell_host.cpp")])
    lb = ctypes.CDLL(out)
    lb.v3_host_neighbors.restype = ctypes.c_int64
    lb.v3_host_neighbors.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    return lb


def _rows(lib, pos, box, order, maxdeg=96):
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    box = np.asarray(box, dtype=np.int64)
    n = pos.shape[0]
    deg = np.zeros(n, dtype=np.int32)
    ids = np.zeros(n * maxdeg, dtype=np.int32)
    lib.v3_host_neighbors(n, pos.ctypes.data, box.ctypes.data, order, maxdeg, deg.ctypes.data, ids.ctypes.data)
    assert (deg >= 0).all(), f"builder failed: {sorted(set(deg[deg < 0].tolist()))}"
    return [ids[i * maxdeg:i * maxdeg + deg[i]].tolist() for i in range(n)]


def _same(lib, pos, box, orders=(0, 1, 2)):
    off, ids = oracle.voronoi3(pos, box)
    want = [ids[off[i]:off[i + 1]].tolist() for i in range(len(pos))]
    for order in orders:
        got = _rows(lib, pos, box, order)
        bad = [i for i in range(len(pos)) if got[i] != want[i]]
        assert not bad, f"order {order}: particle {bad[0]}: {got[bad[0]]} != {want[bad[0]]}"


@pytest.mark.parametrize("n,L,seed", [(2, 1000, 1), (3, 1000, 2), (5, 1000, 3), (8, 500, 4), (20, 2000, 5),
                                      (64, 4096, 6), (400, 1 << 16, 7), (600, 1 << 23, 8)])
def test_random_boxes(lib, n, L, seed):
    rng = np.random.default_rng(seed)
    pos = rng.integers(0, L, size=(n, 3)).astype(np.int32)
    if len({tuple(p) for p in pos}) < n:
        pytest.skip("coincident draw")
    _same(lib, pos, (L, L, L))


def test_anisotropic_box(lib):
    rng = np.random.default_rng(9)
    box = (500, 900, 3000)
    _same(lib, rng.integers(0, box, size=(200, 3)).astype(np.int32), box)


@pytest.mark.parametrize("kind", ["sc", "bcc", "fcc"])
def test_cubic_lattices(lib, kind):
    pos, box = W.cubic_lattice(kind, 4, 1 << 10, offset_q=(1, 2, 3))
    _same(lib, pos, box)


def test_degenerate_grids(lib):
    """A coarse integer grid (many cospherical groups) and a jittered
    lattice (nearly cospherical: the FP32 filter's band is hit often)."""
    rng = np.random.default_rng(10)
    pos = np.unique(rng.integers(0, 8, size=(150, 3)) * 16, axis=0).astype(np.int32)
    _same(lib, pos, (128, 128, 128))
    m, sp = 8, 1 << 12
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3) * sp
    pos = ((g + rng.integers(-2, 3, size=g.shape)) % (m * sp)).astype(np.int32)
    # index order sweeps the lattice plane by plane and can outgrow even the
    # larger cell; the kernel's ring walk visits near sites first
    _same(lib, pos, (m * sp,) * 3, orders=(1, 2))


def _i32(v):
    a = np.ascontiguousarray(v, dtype=np.int32)
    return a, a.ctypes.data


def _side(lib, da, db, dc, de):
    arrs = [_i32(v) for v in (da, db, dc, de)]
    return lib.v3_host_side(*[p for _, p in arrs])


def _setup_predicates(lib):
    lib.v3_host_side.restype = ctypes.c_int
    lib.v3_host_side.argtypes = [ctypes.c_void_p] * 4
    lib.v3_host_vertex.restype = None
    lib.v3_host_vertex.argtypes = [ctypes.c_void_p] * 4


def _random_offsets(rng, m, norm_max):
    """m integer vectors of Euclidean norm below norm_max (and nonzero)."""
    out = []
    while len(out) < m:
        v = rng.integers(-int(norm_max), int(norm_max), size=3)
        if 0 < int(v @ v) < norm_max * norm_max:
            out.append(v)
    return np.array(out, dtype=np.int64)


def test_exact_side_matches_the_oracle_up_to_the_range_limit(lib):
    """sign(d_e.y - |d_e|^2) at the vertex of planes a, b, c: the builder's
    int128 determinant against the oracle's independent 256-bit one, for
    offsets of norm up to 2^24 (the builder's stated range)."""
    _setup_predicates(lib)
    rng = np.random.default_rng(21)
    for norm_max in (1 << 10, 1 << 20, (1 << 24) - 1):
        d = _random_offsets(rng, 4 * 400, norm_max).reshape(400, 4, 3)
        for da, db, dc, de in d:
            if _det_exact(da, db, dc) == 0:
                continue  # planes without a common point
            assert _side(lib, da, db, dc, de) == oracle.voronoi3_side(da, db, dc, de)


def test_exact_zeros_at_large_coordinates(lib):
    """Planes through one point: with y = (2a, 2b, 2c), every offset d at a
    corner of the box [0, 2a] x [0, 2b] x [0, 2c] has d.y = |d|^2, so the
    vertex of any three of them lies exactly on the fourth (sign 0).  Moving
    the fourth offset by one grid unit along an axis gives small values of
    either sign next to large terms; their signs must match the oracle's.
    Corners up to norm sqrt(3) 2^23 < 2^24."""
    _setup_predicates(lib)
    rng = np.random.default_rng(22)
    for _ in range(60):
        a, b, c = (int(x) for x in rng.integers(1 << 20, 1 << 23, size=3))
        corners = [np.array([sx * 2 * a, sy * 2 * b, sz * 2 * c]) for sx in (0, 1) for sy in (0, 1) for sz in (0, 1)
                   if sx or sy or sz]
        idx = rng.choice(len(corners), size=4, replace=False)
        da, db, dc, de = (corners[i] for i in idx)
        if _det_exact(da, db, dc) == 0:
            continue
        assert oracle.voronoi3_side(da, db, dc, de) == 0
        assert _side(lib, da, db, dc, de) == 0
        for k in range(3):
            for step in (-1, 1):
                e2 = de.copy()
                e2[k] += step
                if int(e2 @ e2) >= (1 << 48):
                    continue
                assert _side(lib, da, db, dc, e2) == oracle.voronoi3_side(da, db, dc, e2)


def test_vertex_estimate_error_bound(lib):
    """The FP32 vertex y (d_x.y = |d_x|^2, x = a, b, c) errs by at most
    2^-22 |y_k| per coordinate (the bound the FP32 side filter assumes):
    checked against the exact rational solution, on random and on
    ill-conditioned (nearly coplanar) triples up to the range limit."""
    from fractions import Fraction
    _setup_predicates(lib)
    rng = np.random.default_rng(23)

    def exact(da, db, dc):
        M = [[Fraction(int(x)) for x in r] + [Fraction(int(r @ r))] for r in (da, db, dc)]
        for col in range(3):
            piv = next(r for r in range(col, 3) if M[r][col] != 0)
            M[col], M[piv] = M[piv], M[col]
            for r in range(3):
                if r != col and M[r][col] != 0:
                    f = M[r][col] / M[col][col]
                    M[r] = [x - f * y for x, y in zip(M[r], M[col])]
        return [M[k][3] / M[k][k] for k in range(3)]

    cases = []
    for norm_max in (1 << 12, 1 << 22, (1 << 24) - 1):
        for t in _random_offsets(rng, 3 * 150, norm_max).reshape(150, 3, 3):
            cases.append(t)
    for _ in range(150):  # nearly coplanar: c close to a combination of a and b
        da, db = _random_offsets(rng, 2, 1 << 22)
        dc = (da + db) // 2 + rng.integers(-2, 3, size=3)
        cases.append(np.array([da, db, dc]))
    checked = 0
    for da, db, dc in cases:
        if _det_exact(da, db, dc) == 0:
            continue
        y = np.zeros(3, dtype=np.float32)
        arrs = [_i32(v) for v in (da, db, dc)]
        lib.v3_host_vertex(arrs[0][1], arrs[1][1], arrs[2][1], y.ctypes.data)
        ye = exact(da, db, dc)
        for k in range(3):
            err = abs(Fraction(float(y[k])) - ye[k])
            assert err <= Fraction(1, 1 << 22) * abs(Fraction(float(y[k]))), (da, db, dc, k)
        checked += 1
    assert checked > 500


def _det_exact(a, b, c):
    a, b, c = ([int(x) for x in v] for v in (a, b, c))
    return (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
            a[2] * (b[0] * c[1] - b[1] * c[0]))
