"""GPU parity of the rule variants of Sec. "Metric and topological flocking
models": the metric rule (every particle within r0, 2D and 3D) and the k
nearest neighbors inside a field of view (2D).  Lists are compared with the
oracle's brute force element by element (bit-exact), and each checked step
is teacher-forced against the oracle's FP64 update from the same state
(positions exact, headings within 1e-5 rad)."""
import numpy as np
import pytest

import oracle
from paper_2103_10239_gb300 import vk
from paper_2103_10239_gb300 import workloads as W
from parity import check_step

pytestmark = pytest.mark.gpu


def r0q_of(r0: float, frac_bits: int) -> int:
    """rint(r0 * 2^F), round half to even, from the FP32 value of r0."""
    return int(np.rint(np.float64(np.float32(r0)) * float(1 << frac_bits)))


def metric_lists(box_q, r0q):
    return lambda pos, d: oracle.metric(pos, box_q, r0q)


def fov_lists(box_q, k, fov_cos):
    def f(pos, d):
        ids, cnt = oracle.knn_fov(pos, d, box_q, k, fov_cos)
        off = np.zeros(pos.shape[0] + 1, dtype=np.int64)
        off[1:] = np.cumsum(cnt)
        return off, ids[ids >= 0].astype(np.int32)
    return f


# ---------------------------------------------------------------- metric, 2D

@pytest.mark.parametrize("r0", [0.0, 0.5, 1.0, 2.5, 14.0])
def test_metric_2d_lists_and_steps(r0):
    """N=3000 at density ~1 (L=54, F=16).  r0 = 14 is above a quarter of
    the box, where the square walk hands over to a scan of the replica."""
    w = W.uniform_system(3000, 54.0, 16, 2, input_seed=41, rule="metric", k=0, v0=0.5, eta=0.4)
    r0q = r0q_of(r0, w.frac_bits)
    with vk.from_workload(w, r0=r0) as sim:
        for _ in range(3):
            check_step(sim, w, "metric", lists=metric_lists(w.box_q, r0q))


@pytest.mark.parametrize("occ", [0.5, 2.0, 8.0, 512.0, 4096.0])
def test_metric_2d_lists_do_not_depend_on_the_cell_grid(occ):
    w = W.uniform_system(2500, 50.0, 16, 2, input_seed=43, rule="metric", k=0)
    r0q = r0q_of(1.7, w.frac_bits)
    want = oracle.metric(w.pos_q, w.box_q, r0q)
    with vk.from_workload(w, r0=1.7, cell_occupancy=occ) as sim:
        off, ids = sim.neighbors()
        assert np.array_equal(off, want[0]) and np.array_equal(ids, want[1])


@pytest.mark.parametrize("noise,include_self,advect_new", [("angular", True, False), ("vectorial", False, False),
                                                            ("vectorial", True, True)])
def test_metric_2d_update_modes(noise, include_self, advect_new):
    w = W.uniform_system(2000, 40.0, 16, 2, input_seed=45, rule="metric", k=0, v0=0.5, eta=0.6, noise=noise)
    r0q = r0q_of(1.0, w.frac_bits)
    with vk.from_workload(w, r0=1.0, include_self=int(include_self), advect_new=int(advect_new)) as sim:
        for _ in range(3):
            check_step(sim, w, "metric", lists=metric_lists(w.box_q, r0q), include_self=include_self,
                       advect_new=advect_new)


def test_metric_2d_clustered_flock():
    """Gaussian clusters over a uniform background: dense coarse cells get
    sub-grids, and rows of a few hundred neighbors occur."""
    w = W.clustered_large(n=20000, n_clusters=8, sigma=2.0, seed=47)
    r0q = r0q_of(1.0, w.frac_bits)
    want = oracle.metric(w.pos_q, w.box_q, r0q)
    with vk.from_workload(w, rule="metric", r0=1.0) as sim:
        off, ids = sim.neighbors()
        assert np.array_equal(off, want[0]) and np.array_equal(ids, want[1])
        assert np.diff(off).max() > 100


def test_metric_square_lattice_is_inclusive():
    """Lattice spacing a = 1 (2^16 grid units): r0 = a gives exactly the 4
    axis neighbors (D = r0q^2 counts), just below a none, r0 = sqrt(2) a
    rounds to 92682 grid units, above sqrt(2) a, so 8 neighbors."""
    pos, box = W.square_lattice(8, 1 << 16, 0)
    d = W.random_dirs(pos.shape[0])
    for r0, deg in [(1.0, 4), (0.99999, 0), (float(np.sqrt(2.0)), 8), (2.0, 12)]:
        with vk.Sim.create(pos, d, box, 16, rule="metric", r0=r0) as sim:
            off, ids = sim.neighbors()
            assert np.all(np.diff(off) == deg)
            want = oracle.metric(pos, box, r0q_of(r0, 16))
            assert np.array_equal(ids, want[1])


@pytest.mark.parametrize("n,L,bits", [(2, 4.0, 16), (8, 4.0, 16), (255, 16.0, 12), (257, 16.0, 20)])
def test_metric_ragged_sizes(n, L, bits):
    w = W.uniform_system(n, L, bits, 2, input_seed=n, rule="metric", k=0, v0=0.5, eta=0.4)
    r0q = r0q_of(1.5, bits)
    with vk.from_workload(w, r0=1.5) as sim:
        for _ in range(2):
            check_step(sim, w, "metric", lists=metric_lists(w.box_q, r0q))


def test_metric_run_to_run_bit_identical():
    """The heading sums are exact integers, so two runs agree bit for bit
    (positions, headings and phi), whatever order the cells list particles."""
    w = W.uniform_system(20000, 100.0, 16, 2, input_seed=49, rule="metric", k=0, v0=0.5, eta=0.3)
    out = []
    for _ in range(2):
        with vk.from_workload(w, r0=1.0) as sim:
            sim.step(20)
            p, d, _, _ = sim.state()
            out.append((p, d, sim.order_parameter()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])


# ---------------------------------------------------------------- metric, 3D

@pytest.mark.parametrize("r0", [0.7, 1.3, 2.5])
def test_metric_3d_lists_and_steps(r0):
    w = W.uniform_system(2000, 12.6, 16, 3, input_seed=51, rule="metric", k=0, v0=0.5, eta=0.4,
                         noise="vectorial")
    r0q = r0q_of(r0, w.frac_bits)
    with vk.from_workload(w, r0=r0) as sim:
        for _ in range(3):
            check_step(sim, w, "metric", lists=metric_lists(w.box_q, r0q))


# ------------------------------------------------------- field of view, 2D kNN

@pytest.mark.parametrize("fov_cos", [-1.0, -0.5, 0.0, 0.5, 0.9])
@pytest.mark.parametrize("search", [0, 1])
def test_fov_lists_and_steps(fov_cos, search):
    w = W.uniform_system(3000, 54.0, 16, 2, input_seed=53, rule="knn", k=7, v0=0.5, eta=0.4)
    with vk.from_workload(w, fov=1, fov_cos=fov_cos, knn_search=search) as sim:
        for _ in range(3):
            check_step(sim, w, "knn", lists=fov_lists(w.box_q, 7, fov_cos))


@pytest.mark.parametrize("noise,include_self", [("vectorial", False), ("vectorial", True), ("angular", True)])
def test_fov_update_modes(noise, include_self):
    """A short in-view list changes m, the count Eq. (2) averages over."""
    w = W.uniform_system(2000, 44.0, 16, 2, input_seed=58, rule="knn", k=6, v0=0.5, eta=0.5, noise=noise)
    with vk.from_workload(w, fov=1, fov_cos=0.6, include_self=int(include_self)) as sim:
        for _ in range(3):
            check_step(sim, w, "knn", lists=fov_lists(w.box_q, 6, 0.6), include_self=include_self)


def test_fov_full_circle_is_the_plain_rule():
    w = W.uniform_system(2000, 44.0, 16, 2, input_seed=55, rule="knn", k=7)
    with vk.from_workload(w, fov=1, fov_cos=-1.0) as a, vk.from_workload(w) as b:
        a.step(5)
        b.step(5)
        assert np.array_equal(a.neighbors()[1], b.neighbors()[1])
        assert np.array_equal(a.state()[0], b.state()[0])


def test_fov_zero_width_view_has_short_rows():
    """cos = 1: only particles exactly straight ahead are in view, which on
    the integer grid with FP32 headings is almost nobody; rows are shorter
    than k (empty rows align with nobody: own heading plus noise)."""
    w = W.uniform_system(1500, 38.0, 16, 2, input_seed=57, rule="knn", k=4, v0=0.5, eta=0.4)
    with vk.from_workload(w, fov=1, fov_cos=1.0) as sim:
        off, _ = sim.neighbors()
        assert np.diff(off).max() < 4
        for _ in range(2):
            check_step(sim, w, "knn", lists=fov_lists(w.box_q, 4, 1.0))


def test_fov_on_a_lattice_with_ties():
    """Square lattice with axis-aligned headings: the view boundary passes
    through lattice points and equal distances are everywhere."""
    pos, box = W.square_lattice(9, 1 << 16, 0)
    n = pos.shape[0]
    axes = np.array([[1, 0], [0, 1], [-1, 0], [0, -1]], dtype=np.float32)
    d = axes[np.arange(n) % 4]
    for fov_cos in [0.0, float(np.float32(np.sqrt(0.5))), -0.5]:
        for search in (0, 1):
            with vk.Sim.create(pos, d, box, 16, k=6, fov=1, fov_cos=fov_cos, knn_search=search) as sim:
                off, ids = sim.neighbors()
                want = fov_lists(box, 6, fov_cos)(pos, d)
                assert np.array_equal(off, want[0]) and np.array_equal(ids, want[1])


def test_fov_after_many_steps_with_hints():
    """The radius-first search sizes its square from last step's k-th
    in-view distance; after 30 steps the lists still match brute force."""
    w = W.uniform_system(6000, 77.0, 16, 2, input_seed=59, rule="knn", k=7, v0=0.5, eta=0.2)
    with vk.from_workload(w, fov=1, fov_cos=0.2) as sim:
        sim.step(30)
        check_step(sim, w, "knn", lists=fov_lists(w.box_q, 7, 0.2))


# ------------------------------------------------------------ batched replicas

def test_metric_and_view_in_a_replica_batch():
    """Replicas with their own box and fixed-point resolution: r0q is
    rint(r0 * 2^F) per replica; each replica's lists and one teacher-forced
    step match the oracle, for the metric rule and for a field of view."""
    ws = [W.uniform_system(n, L, F, 2, input_seed=70 + i, rule="metric", k=5, v0=0.5, eta=0.3)
          for i, (n, L, F) in enumerate([(700, 26.0, 16), (1500, 30.0, 12), (300, 15.0, 20)])]
    pos = np.ascontiguousarray(np.concatenate([w.pos_q for w in ws]))
    d = np.ascontiguousarray(np.concatenate([w.dir for w in ws]))
    for params, lists in [(dict(rule="metric", r0=1.3), lambda w: metric_lists(w.box_q, r0q_of(1.3, w.frac_bits))),
                          (dict(rule="knn", k=5, fov=1, fov_cos=0.3), lambda w: fov_lists(w.box_q, 5, 0.3))]:
        with vk.Sim.create_batch([w.n for w in ws], pos, d, [w.box_q for w in ws], [w.frac_bits for w in ws],
                                 eta_r=[w.eta for w in ws], v0=0.5, eta=0.3, **params) as sim:
            for _ in range(2):
                for r, w in enumerate(ws):
                    pos0, d0, _, t0 = sim.state(r)
                    off, ids = sim.neighbors(r)
                    woff, wids = lists(w)(pos0, d0)
                    assert np.array_equal(off, woff) and np.array_equal(ids, wids), (params, r)
                sim.step(1)
