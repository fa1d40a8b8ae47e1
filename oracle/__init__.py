"""CPU oracle for the topological Vicsek hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product path (the CUDA
library and its Python binding) never calls it and never falls back to it.

The numerical work lives in ``vk_oracle.c`` (plain C, FP64 and exact
integers, OpenMP over particles); this module builds it with gcc and wraps it
with ctypes.  ``oracle.brute`` holds small pure-Python references (exact
rational arithmetic) used to pin the C code on tiny inputs.

Functions and the passages of arxiv 2103.10239 they follow:

* :func:`knn` -- k nearest neighbors with no cutoff (Sec. "Metric and
  topological flocking models"), brute force over all pairs.
* :func:`metric` -- all particles within a distance r0 (Sec. "Metric and
  topological flocking models"), brute force over all pairs.
* :func:`knn_fov` -- the k nearest particles inside a field of view (same
  section), brute force over all pairs.
* :func:`voronoi` -- Voronoi neighbors via the Delaunay triangulation's
  empty-circumcircle definition and the Delaunay/Voronoi duality (Sec.
  "Computational tools: Voronoi neighbor lists").
* :func:`voronoi3` -- 3D Voronoi neighbors (same section): each cell by
  exact half-space clipping with the bisectors of the periodic images,
  neighbors sharing a face of positive area, and the cell volumes.
* :func:`vicsek_step` -- Eq. (1) advection and Eq. (2) alignment with noise.
* :func:`order_parameter` -- the polar order |sum n_i|/N.
* :func:`philox4x32_10` -- the counter-based generator the noise is drawn from.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libvk_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
_ERRS = {1: "bad argument", 2: "out of memory", 3: "degenerate input (coincident points)",
         4: "internal error"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with the host gcc (OpenMP on)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.orc_philox4x32_10.restype = None
        lib.orc_knn.argtypes = [ctypes.c_int, ctypes.c_int64, i32p, i64p, ctypes.c_int, i64p,
                                ctypes.c_int64, i32p]
        lib.orc_knn.restype = ctypes.c_int
        lib.orc_voronoi.argtypes = [ctypes.c_int64, i32p, i64p, i64p, i32p, ctypes.c_int64, i64p]
        lib.orc_voronoi.restype = ctypes.c_int
        lib.orc_metric.argtypes = [ctypes.c_int, ctypes.c_int64, i32p, i64p, ctypes.c_int64, i64p, i32p,
                                   ctypes.c_int64, i64p]
        lib.orc_metric.restype = ctypes.c_int
        lib.orc_knn_fov.argtypes = [ctypes.c_int64, i32p, ctypes.POINTER(ctypes.c_float), i64p, ctypes.c_int,
                                    ctypes.c_float, i64p, ctypes.c_int64, i32p, i32p]
        lib.orc_knn_fov.restype = ctypes.c_int
        lib.orc_delaunay_star_triangles.argtypes = [ctypes.c_int64, i32p, i64p, i64p, i32p,
                                                    ctypes.c_int64, i64p]
        lib.orc_delaunay_star_triangles.restype = ctypes.c_int
        lib.orc_orient2d.argtypes = [i64p, i64p, i64p]
        lib.orc_orient2d.restype = ctypes.c_int
        lib.orc_incircle.argtypes = [i64p, i64p, i64p, i64p]
        lib.orc_incircle.restype = ctypes.c_int
        lib.orc_vicsek_step.argtypes = [ctypes.c_void_p, ctypes.c_int64, i32p,
                                        ctypes.POINTER(ctypes.c_float), i64p, i64p, i32p,
                                        ctypes.c_int64, ctypes.c_uint32, i32p,
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]
        lib.orc_vicsek_step.restype = ctypes.c_int
        lib.orc_order_parameter_f32.argtypes = [ctypes.c_int, ctypes.c_int64,
                                                ctypes.POINTER(ctypes.c_float)]
        lib.orc_order_parameter_f32.restype = ctypes.c_double
        lib.orc_order_parameter_f64.argtypes = [ctypes.c_int, ctypes.c_int64,
                                                ctypes.POINTER(ctypes.c_double)]
        lib.orc_order_parameter_f64.restype = ctypes.c_double
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.orc_tissue.argtypes = [ctypes.c_int64, i32p, i64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, f64p, f64p, f64p, f64p]
        lib.orc_tissue.restype = ctypes.c_int
        lib.orc_voronoi3.argtypes = [ctypes.c_int64, i32p, i64p, i64p, ctypes.c_int64, ctypes.c_int32, i32p,
                                     i32p, f64p]
        lib.orc_voronoi3.restype = ctypes.c_int
        lib.orc_voronoi3_side.argtypes = [i64p, i64p, i64p, i64p]
        lib.orc_voronoi3_side.restype = ctypes.c_int
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(rc: int, what: str):
    if rc != ORC_OK:
        raise OracleError(f"{what}: {_ERRS.get(rc, rc)}")


def num_threads() -> int:
    return int(_load().orc_num_threads())


def philox4x32_10(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    """Philox4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    o = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(o, ctypes.c_uint32))
    return o


def _box(box_q, dim) -> np.ndarray:
    b = np.asarray(list(box_q), dtype=np.int64)
    if b.shape != (dim,):
        raise ValueError("box must have one edge per axis")
    return b


def knn(pos_q: np.ndarray, box_q, k: int, query: Optional[np.ndarray] = None) -> np.ndarray:
    """k nearest other particles of each (query) particle, ordered by
    (exact squared minimum-image distance, id).  Returns (nq, k) int32."""
    lib = _load()
    pos = np.ascontiguousarray(pos_q, dtype=np.int32)
    n, dim = pos.shape
    box = _box(box_q, dim)
    if query is None:
        q = None
        nq = n
    else:
        q = np.ascontiguousarray(query, dtype=np.int64)
        nq = q.shape[0]
    out = np.zeros((nq, k), dtype=np.int32)
    rc = lib.orc_knn(dim, n, _ptr(pos, ctypes.c_int32), _ptr(box, ctypes.c_int64), k,
                     None if q is None else _ptr(q, ctypes.c_int64), nq, _ptr(out, ctypes.c_int32))
    _check(rc, "knn")
    return out


def metric(pos_q: np.ndarray, box_q, r0_q: int):
    """Metric neighbors: every other particle at exact squared minimum-image
    distance <= r0_q^2 (grid units).  Returns (offsets int64[n+1], ids
    int32[nnz]), rows sorted by id."""
    lib = _load()
    pos = np.ascontiguousarray(pos_q, dtype=np.int32)
    n, dim = pos.shape
    box = _box(box_q, dim)
    off = np.zeros(n + 1, dtype=np.int64)
    nnz = np.zeros(1, dtype=np.int64)
    rc = lib.orc_metric(dim, n, _ptr(pos, ctypes.c_int32), _ptr(box, ctypes.c_int64), int(r0_q),
                        _ptr(off, ctypes.c_int64), None, 0, _ptr(nnz, ctypes.c_int64))
    _check(rc, "metric (size)")
    ids = np.zeros(max(1, int(nnz[0])), dtype=np.int32)
    rc = lib.orc_metric(dim, n, _ptr(pos, ctypes.c_int32), _ptr(box, ctypes.c_int64), int(r0_q),
                        _ptr(off, ctypes.c_int64), _ptr(ids, ctypes.c_int32), ids.shape[0],
                        _ptr(nnz, ctypes.c_int64))
    _check(rc, "metric")
    return off, ids[: int(nnz[0])]


def knn_fov(pos_q: np.ndarray, dir32: np.ndarray, box_q, k: int, fov_cos: float,
            query: Optional[np.ndarray] = None):
    """k nearest neighbors inside each particle's field of view (2D): the
    offset d must satisfy d.nq >= cq |d| with the heading and the cosine of
    the half-angle rounded to 2^-24.  Returns (ids (nq, k) int32 with -1 past
    the count, count (nq,) int32)."""
    lib = _load()
    pos = np.ascontiguousarray(pos_q, dtype=np.int32)
    d = np.ascontiguousarray(dir32, dtype=np.float32)
    n = pos.shape[0]
    box = _box(box_q, 2)
    if query is None:
        q = None
        nq = n
    else:
        q = np.ascontiguousarray(query, dtype=np.int64)
        nq = q.shape[0]
    out = np.zeros((nq, k), dtype=np.int32)
    cnt = np.zeros(nq, dtype=np.int32)
    rc = lib.orc_knn_fov(n, _ptr(pos, ctypes.c_int32), _ptr(d, ctypes.c_float), _ptr(box, ctypes.c_int64), k,
                         float(np.float32(fov_cos)), None if q is None else _ptr(q, ctypes.c_int64), nq,
                         _ptr(out, ctypes.c_int32), _ptr(cnt, ctypes.c_int32))
    _check(rc, "knn_fov")
    return out, cnt


def voronoi(pos_q: np.ndarray, box_q):
    """Voronoi neighbors (positive-length shared edge) of every particle in a
    periodic square box.  Returns (offsets int64[n+1], ids int32[nnz]), each
    row sorted by id."""
    lib = _load()
    pos = np.ascontiguousarray(pos_q, dtype=np.int32)
    n = pos.shape[0]
    box = _box(box_q, 2)
    off = np.zeros(n + 1, dtype=np.int64)
    nnz = np.zeros(1, dtype=np.int64)
    rc = lib.orc_voronoi(n, _ptr(pos, ctypes.c_int32), _ptr(box, ctypes.c_int64),
                         _ptr(off, ctypes.c_int64), None, 0, _ptr(nnz, ctypes.c_int64))
    _check(rc, "voronoi (size)")
    ids = np.zeros(max(1, int(nnz[0])), dtype=np.int32)
    rc = lib.orc_voronoi(n, _ptr(pos, ctypes.c_int32), _ptr(box, ctypes.c_int64),
                         _ptr(off, ctypes.c_int64), _ptr(ids, ctypes.c_int32), ids.shape[0],
                         _ptr(nnz, ctypes.c_int64))
    _check(rc, "voronoi")
    return off, ids[: int(nnz[0])]


def voronoi3(pos_q: np.ndarray, box_q, query: Optional[np.ndarray] = None, volumes: bool = False):
    """Voronoi neighbors in a periodic 3D box: the particles whose cell shares
    a face of positive area with the cell of each (query) particle.  Returns
    (offsets int64[nq+1], ids int32[nnz]) with rows sorted by id, plus the
    cell volumes in grid units^3 (float64[nq]) when ``volumes``."""
    lib = _load()
    pos = np.ascontiguousarray(pos_q, dtype=np.int32)
    n = pos.shape[0]
    box = _box(box_q, 3)
    q = None if query is None else np.ascontiguousarray(query, dtype=np.int64)
    nq = n if q is None else q.shape[0]
    vol = np.zeros(max(1, nq), dtype=np.float64)
    maxdeg = 64
    while True:
        deg = np.zeros(max(1, nq), dtype=np.int32)
        ids = np.zeros(max(1, nq) * maxdeg, dtype=np.int32)
        rc = lib.orc_voronoi3(n, _ptr(pos, ctypes.c_int32), _ptr(box, ctypes.c_int64),
                              None if q is None else _ptr(q, ctypes.c_int64), nq, maxdeg,
                              _ptr(deg, ctypes.c_int32), _ptr(ids, ctypes.c_int32), _ptr(vol, ctypes.c_double))
        if rc == 1 and nq and int(deg[:nq].max()) > maxdeg:
            maxdeg = int(deg[:nq].max())
            continue
        _check(rc, "voronoi3")
        break
    deg = deg[:nq].astype(np.int64)
    off = np.zeros(nq + 1, dtype=np.int64)
    np.cumsum(deg, out=off[1:])
    rows = ids.reshape(max(1, nq), maxdeg)
    out = np.concatenate([rows[r, : deg[r]] for r in range(nq)]) if nq else np.zeros(0, np.int32)
    out = out.astype(np.int32)
    if volumes:
        return off, out, vol[:nq].copy()
    return off, out


def voronoi3_side(da, db, dc, de) -> int:
    """Sign of d_e.y - |d_e|^2 at the point y where d_x.y = |d_x|^2 for
    x = a, b, c (the exact vertex test of :func:`voronoi3`)."""
    lib = _load()
    arrs = [np.asarray(p, dtype=np.int64).copy() for p in (da, db, dc, de)]
    return int(lib.orc_voronoi3_side(*[_ptr(p, ctypes.c_int64) for p in arrs]))


def delaunay_star_triangles(pos_q: np.ndarray, box_q):
    """Triangles of the periodic Delaunay triangulation touching an original
    point: (coords int64 (T,3,2) in tiled coordinates, ids int32 (T,3))."""
    lib = _load()
    pos = np.ascontiguousarray(pos_q, dtype=np.int32)
    n = pos.shape[0]
    box = _box(box_q, 2)
    cap = 12 * n + 64
    coords = np.zeros((cap, 3, 2), dtype=np.int64)
    tids = np.zeros((cap, 3), dtype=np.int32)
    nt = np.zeros(1, dtype=np.int64)
    rc = lib.orc_delaunay_star_triangles(n, _ptr(pos, ctypes.c_int32), _ptr(box, ctypes.c_int64),
                                         _ptr(coords, ctypes.c_int64), _ptr(tids, ctypes.c_int32),
                                         cap, _ptr(nt, ctypes.c_int64))
    _check(rc, "delaunay_star_triangles")
    t = int(nt[0])
    return coords[:t], tids[:t]


def tissue(pos_q: np.ndarray, box_q, frac_bits: int, KA: float, KP: float, A0: float, P0: float,
           forces: bool = True):
    """Voronoi tissue model in length units (grid unit = 2^-F): cell areas
    and perimeters, the energy of Eq. (vmEnergy) and the forces -dE/dr_i.
    Returns (area (n,), perimeter (n,), energy, force (n, 2) or None)."""
    lib = _load()
    pos = np.ascontiguousarray(pos_q, dtype=np.int32)
    n = pos.shape[0]
    box = _box(box_q, 2)
    area = np.zeros(n, dtype=np.float64)
    perim = np.zeros(n, dtype=np.float64)
    force = np.zeros((n, 2), dtype=np.float64) if forces else None
    e = np.zeros(1, dtype=np.float64)
    f64 = ctypes.POINTER(ctypes.c_double)
    rc = lib.orc_tissue(n, _ptr(pos, ctypes.c_int32), _ptr(box, ctypes.c_int64), 2.0 ** -frac_bits, float(KA),
                        float(KP), float(A0), float(P0), _ptr(area, ctypes.c_double), _ptr(perim, ctypes.c_double),
                        _ptr(force, ctypes.c_double) if forces else ctypes.cast(None, f64), _ptr(e, ctypes.c_double))
    _check(rc, "tissue")
    return area, perim, float(e[0]), force


def orient2d(a, b, c) -> int:
    lib = _load()
    arrs = [np.asarray(p, dtype=np.int64).copy() for p in (a, b, c)]
    return int(lib.orc_orient2d(*[_ptr(p, ctypes.c_int64) for p in arrs]))


def incircle(a, b, c, d) -> int:
    lib = _load()
    arrs = [np.asarray(p, dtype=np.int64).copy() for p in (a, b, c, d)]
    return int(lib.orc_incircle(*[_ptr(p, ctypes.c_int64) for p in arrs]))


class _Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("frac_bits", ctypes.c_int32), ("noise", ctypes.c_int32),
                ("include_self", ctypes.c_int32), ("advect_new", ctypes.c_int32),
                ("v0", ctypes.c_float), ("dt", ctypes.c_float), ("eta", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


def csr_from_dense(nbr: np.ndarray):
    """(n, k) neighbor table -> CSR (offsets, ids)."""
    n, k = nbr.shape
    off = np.arange(n + 1, dtype=np.int64) * k
    return off, np.ascontiguousarray(nbr, dtype=np.int32).ravel()


def vicsek_step(pos_q: np.ndarray, dir32: np.ndarray, box_q, nb_off: np.ndarray,
                nb_ids: np.ndarray, *, frac_bits: int, v0: float, dt: float, eta: float,
                seed: int, step: int, replica: int = 0, noise: str = "angular",
                include_self: bool = False, advect_new: bool = False):
    """One update from the state at `step` (positions, FP32 headings) with the
    given neighbor CSR.  Returns (pos int32, dir float64, theta float64|None)."""
    lib = _load()
    pos = np.ascontiguousarray(pos_q, dtype=np.int32)
    d32 = np.ascontiguousarray(dir32, dtype=np.float32)
    n, dim = pos.shape
    box = _box(box_q, dim)
    off = np.ascontiguousarray(nb_off, dtype=np.int64)
    ids = np.ascontiguousarray(nb_ids, dtype=np.int32)
    if ids.size == 0:
        ids = np.zeros(1, dtype=np.int32)
    prm = _Params(dim, frac_bits, 0 if noise == "angular" else 1, int(include_self),
                  int(advect_new), float(np.float32(v0)), float(np.float32(dt)),
                  float(np.float32(eta)), int(seed) & ((1 << 64) - 1))
    pout = np.zeros_like(pos)
    dout = np.zeros((n, dim), dtype=np.float64)
    tout = np.zeros(n, dtype=np.float64)
    rc = lib.orc_vicsek_step(ctypes.byref(prm), n, _ptr(pos, ctypes.c_int32),
                             _ptr(d32, ctypes.c_float), _ptr(box, ctypes.c_int64),
                             _ptr(off, ctypes.c_int64), _ptr(ids, ctypes.c_int32), int(step),
                             int(replica) & 0xFFFFFFFF, _ptr(pout, ctypes.c_int32),
                             _ptr(dout, ctypes.c_double),
                             _ptr(tout, ctypes.c_double) if dim == 2 else None)
    _check(rc, "vicsek_step")
    return pout, dout, (tout if dim == 2 else None)


def order_parameter(dirs: np.ndarray) -> float:
    lib = _load()
    d = np.ascontiguousarray(dirs)
    n, dim = d.shape
    if d.dtype == np.float32:
        return float(lib.orc_order_parameter_f32(dim, n, _ptr(d, ctypes.c_float)))
    d = np.ascontiguousarray(d, dtype=np.float64)
    return float(lib.orc_order_parameter_f64(dim, n, _ptr(d, ctypes.c_double)))


def neighbors(pos_q: np.ndarray, box_q, rule: str, k: int = 7):
    """Neighbor CSR in canonical order for either rule."""
    if rule == "knn":
        return csr_from_dense(knn(pos_q, box_q, k))
    if rule == "voronoi":
        return voronoi3(pos_q, box_q) if np.asarray(pos_q).shape[1] == 3 else voronoi(pos_q, box_q)
    raise ValueError(rule)
