"""GPU parity of the k-nearest-neighbor rule (Sec. "Metric and topological
flocking models"): lists bit-exact against the brute-force oracle, and one
teacher-forced Vicsek step per checked step."""
import math

import numpy as np
import pytest

import oracle
from paper_2103_10239_gb300 import vk
from paper_2103_10239_gb300 import workloads as W
from parity import check_step, angle_between, PHI_TOL

pytestmark = pytest.mark.gpu


def _knn_lists(sim, k):
    off, ids = sim.neighbors()
    return ids.reshape(-1, k)


def test_topological_small_50_steps_teacher_forced():
    """N=2048, L=45.25, F=16, k=7, eta=0.3: lists every step, headings
    within 1e-5 rad per step, positions exact, phi within 1e-6."""
    w = W.topological_small()
    with vk.from_workload(w) as sim:
        worst = 0.0
        for t in range(w.steps):
            _, _, od, e = check_step(sim, w, "knn")
            worst = max(worst, e)
        phi = sim.order_parameter()
        assert phi.shape[0] == w.steps
        _, d, _, _ = sim.state()
        assert abs(phi[-1] - oracle.order_parameter(d)) < PHI_TOL
        assert worst < 1e-5


@pytest.mark.parametrize("n,L,bits,k", [(8, 4.0, 16, 7), (255, 16.0, 16, 7), (257, 16.0, 16, 6),
                                         (1000, 31.6, 20, 12), (3000, 55.0, 10, 1), (600, 24.5, 16, 16),
                                         (700, 26.0, 16, 32), (33, 3.0, 12, 8)])
def test_ragged_sizes_and_k(n, L, bits, k):
    w = W.uniform_system(n, L, bits, 2, input_seed=n + k, rule="knn", k=k, v0=0.5, eta=0.4)
    with vk.from_workload(w) as sim:
        for _ in range(3):
            check_step(sim, w, "knn")


@pytest.mark.parametrize("occ", [0.3, 1.0, 2.0, 4.0, 9.0, 40.0, 512.0, 4096.0])
def test_lists_do_not_depend_on_the_cell_grid(occ):
    w = W.uniform_system(2500, 50.0, 16, 2, input_seed=3, rule="knn", k=7)
    want = oracle.knn(w.pos_q, w.box_q, 7)
    with vk.from_workload(w, cell_occupancy=occ) as sim:
        pos, _, _, _ = sim.state()
        assert np.array_equal(pos, w.pos_q)
        assert np.array_equal(_knn_lists(sim, 7), want)


@pytest.mark.parametrize("m,a,k", [(6, 1 << 16, 4), (6, 1 << 16, 7), (6, 1 << 16, 8), (9, 1000, 7),
                                   (17, 65536, 12), (3, 10, 8)])
def test_square_lattice_ties(m, a, k):
    pos, box = W.square_lattice(m, a, 0)
    d = W.random_dirs(pos.shape[0])
    with vk.Sim.create(pos, d, box, 16, k=k) as sim:
        assert np.array_equal(_knn_lists(sim, k), oracle.knn(pos, box, k))


def test_translation_invariance_on_gpu():
    w = W.uniform_system(3000, 54.0, 16, 2, input_seed=5, rule="knn", k=7)
    base = oracle.knn(w.pos_q, w.box_q, 7)
    for shift in [(0, 0), (12345, 777), (w.box_q[0] - 1, 1), (w.box_q[0] // 2, w.box_q[1] // 2)]:
        p = np.mod(w.pos_q.astype(np.int64) + np.array(shift), w.box_q[0]).astype(np.int32)
        with vk.Sim.create(p, w.dir, w.box_q, 16, k=7) as sim:
            assert np.array_equal(_knn_lists(sim, 7), base)


@pytest.mark.parametrize("occ", [0.5, 2.0, 8.0, 40.0, 512.0, 4096.0, 32768.0])
def test_clustered_lists_for_any_coarse_occupancy(occ):
    """Dense coarse cells are split into sub-grids; the lists must not
    depend on how the two-level grid is cut (up to a single coarse cell with
    a 64 x 64 sub-grid)."""
    w = W.clustered_large(n=1 << 15)
    want = oracle.knn(w.pos_q, w.box_q, 7)
    with vk.from_workload(w, cell_occupancy=occ) as sim:
        assert np.array_equal(_knn_lists(sim, 7), want)
        sim.step(1)
        check_step(sim, w, "knn")


def test_clustered_density_contrast():
    w = W.clustered_large(n=1 << 15)
    with vk.from_workload(w) as sim:
        for _ in range(2):
            check_step(sim, w, "knn")


@pytest.mark.parametrize("occ,steps", [(None, 2), (2048.0, 40)])
def test_full_scale_clustered_sampled_parity(occ, steps):
    """N = 2^22 (the benchmark workload): sampled particles against brute
    force over all N, plus a teacher-forced step on the same sample; with the
    library's default grid, and in the benchmark's launch configuration
    (2048 particles per coarse cell) on the clumped state after 40 steps."""
    w = W.clustered_large()
    rng = np.random.default_rng(0)
    with vk.from_workload(w, **({} if occ is None else {"cell_occupancy": occ})) as sim:
        sim.step(steps)
        pos0, d0, _, t0 = sim.state()
        off, ids = sim.neighbors()
        q = np.sort(rng.choice(w.n, 1024, replace=False))
        want = oracle.knn(pos0, w.box_q, 7, query=q)
        assert np.array_equal(ids.reshape(-1, 7)[q], want)
        sim.step(1)
        pos1, d1, _, _ = sim.state()
        # the oracle's update of particle i reads only row i of the lists, so
        # rows outside the (verified) sample may come from the GPU; only the
        # sampled rows are compared
        full_off, full_ids = oracle.csr_from_dense(ids.reshape(-1, 7))
        op, od, _ = oracle.vicsek_step(pos0, d0, w.box_q, full_off, full_ids, frac_bits=20, v0=w.v0,
                                       dt=w.dt, eta=w.eta, seed=w.seed, step=t0)
        assert np.array_equal(pos1[q], op[q])
        assert angle_between(d1[q], od[q]).max() <= 1e-5


def test_3d_knn_vectorial():
    w = W.uniform_system(900, 9.65, 16, 3, input_seed=4, rule="knn", k=7, noise="vectorial", eta=0.2)
    with vk.from_workload(w) as sim:
        for _ in range(3):
            check_step(sim, w, "knn")


@pytest.mark.parametrize("n,L,k", [(40, 3.4, 7), (200, 5.8, 7), (700, 8.9, 16), (1500, 11.4, 32), (3000, 14.4, 1)])
def test_3d_radius_first_steps(n, L, k):
    """The 3D step searches the hinted cube first (the ring walk serves what
    the cube cannot: tiny boxes, missed squares); several teacher-forced steps
    so that the hints are in use."""
    w = W.uniform_system(n, L, 16, 3, input_seed=n + k, rule="knn", k=k, noise="vectorial", eta=0.3)
    with vk.from_workload(w) as sim:
        for _ in range(4):
            check_step(sim, w, "knn")


def test_3d_cubic_lattice_ties():
    """Equal distances everywhere: the cube keeps the (D, id) order exactly."""
    m, a = 6, 1 << 16
    i, j, l = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    pos = np.stack([i.ravel() * a, j.ravel() * a, l.ravel() * a], axis=1).astype(np.int32)
    box = (m * a,) * 3
    d = W.random_dirs(pos.shape[0], dim=3)
    for k in (6, 7, 18, 19):
        w = W.Workload(name="lattice3", dim=3, pos_q=pos, dir=d, theta=None, box_q=box, frac_bits=16,
                       rule="knn", k=k, v0=0.0, dt=1.0, eta=0.2, noise="vectorial")
        with vk.from_workload(w) as sim:
            for _ in range(3):
                check_step(sim, w, "knn")


def test_3d_full_size_sampled():
    w = W.knn_3d()
    rng = np.random.default_rng(1)
    with vk.from_workload(w) as sim:
        sim.step(1)
        pos0, _, _, _ = sim.state()
        off, ids = sim.neighbors()
        q = np.sort(rng.choice(w.n, 512, replace=False))
        assert np.array_equal(ids.reshape(-1, 7)[q], oracle.knn(pos0, w.box_q, 7, query=q))


def test_theta_input_matches_dir_input():
    w = W.uniform_system(500, 22.0, 16, 2, input_seed=9, rule="knn", k=7)
    with vk.from_workload(w, heading_kind="theta") as sim:
        _, d, th, _ = sim.state()
    assert angle_between(d, w.dir).max() < 1e-6
    diff = np.abs(((th.astype(np.float64) - w.theta + math.pi) % (2 * math.pi)) - math.pi)
    assert diff.max() < 1e-6


def test_set_state_reports_bad_inputs():
    """vk_set_state reports positions outside the box and non-finite
    headings; a valid call afterwards restores a state that matches the
    oracle (the status word is sticky, so a new simulation is used)."""
    w = W.uniform_system(300, 17.0, 16, 2, input_seed=8, rule="knn", k=7)
    bad = w.pos_q.copy()
    bad[7, 1] = -5
    with vk.from_workload(w) as sim:
        with pytest.raises(vk.VKError) as e:
            sim.set_state(bad, w.dir)
        assert e.value.status == vk.VK_ERR_RANGE
    d = w.dir.copy()
    d[2, 0] = np.inf
    with vk.from_workload(w) as sim:
        with pytest.raises(vk.VKError) as e:
            sim.set_state(w.pos_q, d)
        assert e.value.status == vk.VK_ERR_ARG
    with vk.from_workload(w) as sim:
        sim.step(3)
        sim.set_state(w.pos_q, w.dir, step=0)
        assert np.array_equal(_knn_lists(sim, 7), oracle.knn(w.pos_q, w.box_q, 7))
        check_step(sim, w, "knn")


def test_input_errors():
    w = W.uniform_system(100, 10.0, 16, 2, input_seed=1)
    bad = w.pos_q.copy()
    bad[5, 0] = w.box_q[0]
    with pytest.raises(vk.VKError) as e:
        vk.Sim.create(bad, w.dir, w.box_q, 16, k=7)
    assert e.value.status == vk.VK_ERR_RANGE
    d = w.dir.copy()
    d[3, 1] = np.nan
    with pytest.raises(vk.VKError) as e:
        vk.Sim.create(w.pos_q, d, w.box_q, 16, k=7)
    assert e.value.status == vk.VK_ERR_ARG
