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
