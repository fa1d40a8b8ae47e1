"""Thin Python binding of libvk_nm (the C ABI of ``include/vk.h``).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Arrays may be numpy arrays (host memory) or torch tensors (host or
device); they are passed to the library as raw pointers.  If the compiled
library is missing this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libvk_nm.so")

VK_OK, VK_ERR_ARG, VK_ERR_CUDA, VK_ERR_OOM, VK_ERR_CAPACITY, VK_ERR_RANGE, VK_ERR_DEGENERATE, \
    VK_ERR_TIMEOUT, VK_ERR_STATE = range(9)
VK_RULE_KNN, VK_RULE_VORONOI, VK_RULE_METRIC = 0, 1, 2
VK_NOISE_ANGULAR, VK_NOISE_VECTORIAL = 0, 1
VK_SUM_PLAIN, VK_SUM_COMPENSATED, VK_SUM_FP64 = 0, 1, 2
VK_HEADING_DIR, VK_HEADING_THETA = 0, 1
PHASES = ("search_update", "build", "scatter", "load_sort", "export", "search_deferred")


class VKError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


class vk_box(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("frac_bits", ctypes.c_int32), ("box_q", ctypes.c_uint32 * 3)]


class vk_params(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_int32), ("k", ctypes.c_int32), ("v0", ctypes.c_float),
                ("dt", ctypes.c_float), ("eta", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("noise", ctypes.c_int32), ("include_self", ctypes.c_int32),
                ("advect_new", ctypes.c_int32), ("sum_mode", ctypes.c_int32),
                ("cell_occupancy", ctypes.c_float), ("phi_capacity", ctypes.c_int32),
                ("knn_search", ctypes.c_int32), ("search_halo", ctypes.c_float),
                ("search_halo_step", ctypes.c_float), ("replica_offset", ctypes.c_int32),
                ("r0", ctypes.c_float), ("fov", ctypes.c_int32), ("fov_cos", ctypes.c_float),
                ("voronoi_rebuild", ctypes.c_int32), ("voronoi3_kernel", ctypes.c_int32)]


class vk_info(ctypes.Structure):
    _fields_ = [("n_total", ctypes.c_int64), ("n_rep", ctypes.c_int32), ("dim", ctypes.c_int32),
                ("n_cells", ctypes.c_int64), ("step", ctypes.c_int64),
                ("kernels_per_step", ctypes.c_int32), ("rule", ctypes.c_int32), ("k", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None

_SIGS = {
    "vk_default_params": (None, [ctypes.POINTER(vk_params)]),
    "vk_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                               ctypes.POINTER(vk_box), ctypes.POINTER(vk_params), ctypes.c_void_p,
                               ctypes.POINTER(ctypes.c_void_p)]),
    "vk_batch_init": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int32, ctypes.POINTER(vk_box), ctypes.c_void_p,
                                     ctypes.POINTER(vk_params), ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_void_p)]),
    "vk_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "vk_get_neighbors": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "vk_get_order_parameter": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "vk_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "vk_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int64]),
    "vk_get_tissue": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "vk_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "vk_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "vk_status_string": (ctypes.c_char_p, [ctypes.c_int32]),
    "vk_destroy": (None, [ctypes.c_void_p]),
    "vk_set_graph_steps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "vk_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "vk_get_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32)]),
    "vk_phase_name": (ctypes.c_char_p, [ctypes.c_int32]),
    "vk_get_search_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_double)]),
    "vk_get_search_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int32)]),
    "vk_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(vk_info)]),
    "vk_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_float)]),
    "vk_autotune_forget": (None, []),
    "vk_knn_lists_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(vk_box),
                                            ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
}

NOALLOC_MAX_N = 65536


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load the compiled library (fails loudly when it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libvk_nm is not built ({p} missing); run __graft_entry__.build() "
                               "or python -m paper_2103_10239_gb300._build")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        if path is None:
            _lib = lib
        return lib


def _ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check(rc: int, handle=None):
    if rc != VK_OK:
        msg = load().vk_last_error(handle)
        raise VKError(rc, (msg or b"").decode() or load().vk_status_string(rc).decode())


def default_params(**kw) -> vk_params:
    p = vk_params()
    load().vk_default_params(ctypes.byref(p))
    for key, val in kw.items():
        if key == "rule" and isinstance(val, str):
            val = {"knn": VK_RULE_KNN, "voronoi": VK_RULE_VORONOI, "metric": VK_RULE_METRIC}[val]
        if key == "noise" and isinstance(val, str):
            val = {"angular": VK_NOISE_ANGULAR, "vectorial": VK_NOISE_VECTORIAL}[val]
        if key == "sum_mode" and isinstance(val, str):
            val = {"plain": VK_SUM_PLAIN, "compensated": VK_SUM_COMPENSATED, "fp64": VK_SUM_FP64}[val]
        setattr(p, key, val)
    return p


def make_box(box_q: Sequence[int], frac_bits: int) -> vk_box:
    b = vk_box()
    b.dim = len(box_q)
    b.frac_bits = frac_bits
    for a, v in enumerate(box_q):
        b.box_q[a] = int(v)
    return b


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Sim:
    """One simulation handle (one or more replicas)."""

    def __init__(self, handle: int, n_r: Sequence[int], dim: int, params: vk_params):
        self._h = ctypes.c_void_p(handle)
        self.n_r = [int(x) for x in n_r]
        self.dim = dim
        self.params = params

    # -- construction -----------------------------------------------------
    @classmethod
    def create(cls, pos_q, heading, box_q: Sequence[int], frac_bits: int, heading_kind: str = "dir",
               stream=None, **params) -> "Sim":
        """vk_init: pos_q (N, dim) int32, heading (N, dim) float32 unit vectors
        or (N,) float32 angles (heading_kind="theta")."""
        lib = load()
        prm = default_params(**params)
        box = make_box(box_q, frac_bits)
        n = int(pos_q.shape[0])
        out = ctypes.c_void_p()
        kind = VK_HEADING_THETA if heading_kind == "theta" else VK_HEADING_DIR
        rc = lib.vk_init(_ptr(pos_q), _ptr(heading), kind, n, ctypes.byref(box), ctypes.byref(prm),
                         _stream_handle(stream), ctypes.byref(out))
        _check(rc, None)
        return cls(out.value, [n], len(box_q), prm)

    @classmethod
    def create_batch(cls, n_r: Sequence[int], pos_q, heading, boxes: Sequence[Sequence[int]],
                     frac_bits: Sequence[int], eta_r=None, heading_kind: str = "dir", stream=None,
                     **params) -> "Sim":
        """vk_batch_init: replicas concatenated in pos_q / heading."""
        lib = load()
        prm = default_params(**params)
        nrep = len(n_r)
        arr = (vk_box * nrep)()
        for r in range(nrep):
            arr[r] = make_box(boxes[r], frac_bits[r])
        nr = np.ascontiguousarray(n_r, dtype=np.int64)
        eta = None if eta_r is None else np.ascontiguousarray(eta_r, dtype=np.float32)
        out = ctypes.c_void_p()
        kind = VK_HEADING_THETA if heading_kind == "theta" else VK_HEADING_DIR
        rc = lib.vk_batch_init(nrep, _ptr(nr), _ptr(pos_q), _ptr(heading), kind, arr, _ptr(eta),
                               ctypes.byref(prm), _stream_handle(stream), ctypes.byref(out))
        _check(rc, None)
        return cls(out.value, list(nr), len(boxes[0]), prm)

    # -- the hot path ------------------------------------------------------
    def step(self, n: int = 1):
        _check(load().vk_step(self._h, int(n)), self._h)

    def sync(self):
        _check(load().vk_sync(self._h), self._h)

    # -- observables -------------------------------------------------------
    def neighbors(self, replica: int = 0):
        """(offsets int64[n+1], ids int32[nnz]) of the current positions."""
        lib = load()
        n = self.n_r[replica]
        off = np.zeros(n + 1, dtype=np.int64)
        need = ctypes.c_int64(0)
        _check(lib.vk_get_neighbors(self._h, replica, _ptr(off), None, 0, ctypes.byref(need)), self._h)
        ids = np.zeros(max(1, need.value), dtype=np.int32)
        _check(lib.vk_get_neighbors(self._h, replica, _ptr(off), _ptr(ids), ids.shape[0],
                                    ctypes.byref(need)), self._h)
        return off, ids[: need.value]

    def tissue(self, KA: float, KP: float, A0: float, P0: float, replica: int = 0, forces: bool = True):
        """vk_get_tissue: Voronoi cell areas and perimeters, the energy of
        Eq. (vmEnergy) and the forces -dE/dr_i of the current positions, by
        id, in length units.  Returns (area, perimeter, energy, force|None)."""
        n = self.n_r[replica]
        area = np.zeros(n, dtype=np.float64)
        perim = np.zeros(n, dtype=np.float64)
        force = np.zeros((n, 2), dtype=np.float64) if forces else None
        e = np.zeros(1, dtype=np.float64)
        _check(load().vk_get_tissue(self._h, replica, float(KA), float(KP), float(A0), float(P0),
                                    area.ctypes.data, perim.ctypes.data,
                                    force.ctypes.data if forces else None, e.ctypes.data), self._h)
        return area, perim, float(e[0]), force

    def order_parameter(self, replica: int = 0, max_values: int = 1 << 20) -> np.ndarray:
        lib = load()
        cnt = ctypes.c_int64(0)
        buf = np.zeros(max_values, dtype=np.float64)
        _check(lib.vk_get_order_parameter(self._h, replica, _ptr(buf), max_values, ctypes.byref(cnt)),
               self._h)
        return buf[: cnt.value].copy()

    def state(self, replica: int = 0):
        """(pos_q int32 (n,dim), dir float32 (n,dim), theta float32 (n,) | None, step)."""
        lib = load()
        n = self.n_r[replica]
        pos = np.zeros((n, self.dim), dtype=np.int32)
        d = np.zeros((n, self.dim), dtype=np.float32)
        th = np.zeros(n, dtype=np.float32) if self.dim == 2 else None
        st = ctypes.c_int64(0)
        _check(lib.vk_get_state(self._h, replica, _ptr(pos), _ptr(d), _ptr(th), ctypes.byref(st)),
               self._h)
        return pos, d, th, st.value

    def get_state_into(self, replica: int, pos_q, dirs, theta=None) -> int:
        st = ctypes.c_int64(0)
        _check(load().vk_get_state(self._h, replica, _ptr(pos_q), _ptr(dirs), _ptr(theta),
                                   ctypes.byref(st)), self._h)
        return st.value

    def set_state(self, pos_q, dirs, step: int = -1, replica: int = 0):
        _check(load().vk_set_state(self._h, replica, _ptr(pos_q), _ptr(dirs), int(step)), self._h)

    def info(self) -> vk_info:
        inf = vk_info()
        _check(load().vk_get_info(self._h, ctypes.byref(inf)), self._h)
        return inf

    # -- runtime controls --------------------------------------------------
    def set_graph_steps(self, n: int):
        _check(load().vk_set_graph_steps(self._h, int(n)), self._h)

    def set_profiling(self, on: bool, counters: bool = False):
        level = (2 if counters else 1) if on else 0
        _check(load().vk_set_profiling(self._h, level), self._h)

    def profile(self) -> dict:
        lib = load()
        ms = np.zeros(8, dtype=np.float64)
        la = np.zeros(8, dtype=np.int64)
        nph = ctypes.c_int32(0)
        _check(lib.vk_get_profile(self._h, _ptr(ms), _ptr(la), 8, ctypes.byref(nph)), self._h)
        return {lib.vk_phase_name(p).decode(): (float(ms[p]), int(la[p])) for p in range(nph.value)}

    def search_stats(self) -> dict:
        """Mean candidates / runs per particle update while tracing was on."""
        c = ctypes.c_double(0.0)
        r = ctypes.c_double(0.0)
        m = ctypes.c_int64(0)
        f = ctypes.c_double(0.0)
        _check(load().vk_get_search_stats(self._h, ctypes.byref(c), ctypes.byref(r), ctypes.byref(m),
                                          ctypes.byref(f)), self._h)
        return {"mean_candidates": c.value, "mean_runs": r.value, "max_candidates": m.value,
                "split_fraction": f.value}

    SEARCH_COUNTERS = ("candidates", "runs_or_squares", "max_candidates", "updates", "split_or_walked",
                       "rf_squares", "rf_runs", "rf_candidates", "rf_cells", "rf_hits", "rf_walk_wide",
                       "rf_walk_full", "rf_walk_tie", "rf_walk_few")

    def search_counters(self) -> dict:
        """Raw totals of the search counters while tracing at level 2."""
        vals = np.zeros(len(self.SEARCH_COUNTERS), dtype=np.int64)
        n = ctypes.c_int32(0)
        _check(load().vk_get_search_counters(self._h, vals.ctypes.data, len(vals), ctypes.byref(n)), self._h)
        return dict(zip(self.SEARCH_COUNTERS, (int(v) for v in vals)))

    def autotune(self, candidates: Sequence[float], trial_steps: int = 3) -> float:
        c = np.ascontiguousarray(candidates, dtype=np.float32)
        best = ctypes.c_float(0.0)
        _check(load().vk_autotune(self._h, _ptr(c), c.shape[0], int(trial_steps), ctypes.byref(best)),
               self._h)
        return float(best.value)

    def close(self):
        if self._h is not None and self._h.value:
            load().vk_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def autotune_forget() -> None:
    """vk_autotune_forget: drop the occupancies vk_autotune chose in this process."""
    load().vk_autotune_forget()


def knn_lists_noalloc(pos_q, box_q, frac_bits: int, k: int, out_ids, dev_status=None, stream=None) -> None:
    """vk_knn_lists_noalloc: kNN lists of device-resident points into a
    caller-provided device buffer, using only the library's static scratch
    (no device allocation).  Asynchronous on ``stream``."""
    box = make_box(box_q, frac_bits)
    rc = load().vk_knn_lists_noalloc(_ptr(pos_q), int(pos_q.shape[0]), ctypes.byref(box), int(k), _ptr(out_ids),
                                     _ptr(dev_status), _stream_handle(stream))
    if rc != VK_OK:
        raise VKError(rc, load().vk_status_string(rc).decode())


def from_workload(w, stream=None, heading_kind: str = "dir", **over) -> Sim:
    """Create a Sim from a :class:`workloads.Workload`."""
    params = dict(rule=w.rule, k=max(1, w.k), v0=w.v0, dt=w.dt, eta=w.eta, seed=w.seed, noise=w.noise)
    params.update(over)
    head = w.theta if heading_kind == "theta" else w.dir
    return Sim.create(np.ascontiguousarray(w.pos_q), np.ascontiguousarray(head), w.box_q, w.frac_bits,
                      heading_kind=heading_kind, stream=stream, **params)


def batch_from_workloads(ws, stream=None, **over) -> Sim:
    params = dict(rule=ws[0].rule, k=max(1, ws[0].k), v0=ws[0].v0, dt=ws[0].dt, eta=ws[0].eta,
                  seed=ws[0].seed, noise=ws[0].noise)
    params.update(over)
    pos = np.ascontiguousarray(np.concatenate([w.pos_q for w in ws]))
    d = np.ascontiguousarray(np.concatenate([w.dir for w in ws]))
    return Sim.create_batch([w.n for w in ws], pos, d, [w.box_q for w in ws], [w.frac_bits for w in ws],
                            eta_r=[w.eta for w in ws], stream=stream, **params)
