"""GPU parity of the Voronoi tissue model (Sec. "Geometric models of dense
tissue", Eq. vmEnergy; Sec. "Voronoi model forces") against the oracle:
cell areas and perimeters, the energy and the forces -dE/dr_i.  The GPU
builds the cells with the Voronoi rule's exact clipper and differentiates
the circumcenters in the paper's (c, d, beta d, gamma d) form; the oracle
takes an exact Delaunay triangulation and differentiates the closed-form
circumcenter directly.  Both are FP64: the tolerance is relative 1e-9 on
areas, perimeters and energy, and 1e-7 of the largest force on forces."""
import numpy as np
import pytest

import oracle
from paper_2103_10239_gb300 import vk
from paper_2103_10239_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PARAMS = [(1.0, 1.0, 1.0, 3.8), (2.0, 0.5, 0.9, 3.4), (0.0, 1.0, 0.0, 3.2)]


def _compare(sim, pos, box, F, KA, KP, A0, P0):
    a, p, e, f = sim.tissue(KA, KP, A0, P0)
    oa, op, oe, of = oracle.tissue(pos, box, F, KA, KP, A0, P0)
    assert np.allclose(a, oa, rtol=1e-9, atol=0)
    assert np.allclose(p, op, rtol=1e-9, atol=0)
    assert e == pytest.approx(oe, rel=1e-9, abs=1e-12)
    scale = max(np.abs(of).max(), 1e-6)  # forces that vanish by symmetry: compare against 1e-13 absolute
    assert np.abs(f - of).max() <= 1e-7 * scale
    return a, p, e, f


@pytest.mark.parametrize("KA,KP,A0,P0", PARAMS)
def test_uniform_tissue(KA, KP, A0, P0):
    w = W.uniform_system(3000, 54.0, 16, 2, input_seed=61, rule="voronoi", k=0)
    with vk.from_workload(w) as sim:
        _compare(sim, w.pos_q, w.box_q, w.frac_bits, KA, KP, A0, P0)


def test_lattice_forces_vanish():
    pos, box = W.stretched_hex_lattice(16, 20, 65536, 56756)
    d = W.random_dirs(pos.shape[0])
    with vk.Sim.create(pos, d, box, 16, rule="voronoi") as sim:
        a, p, e, f = _compare(sim, pos, box, 16, 1.0, 1.0, 1.0, 3.8)
        assert np.abs(f).max() < 1e-11
        assert np.ptp(a) == 0.0 or np.ptp(a) < 1e-14


@pytest.mark.parametrize("seed,n,L", [(1, 5, 3.0), (2, 9, 4.0), (3, 30, 6.0)])
def test_tiny_boxes(seed, n, L):
    """Cells bounded by the particle's own periodic images."""
    w = W.uniform_system(n, L, 16, 2, input_seed=seed, rule="voronoi", k=0)
    with vk.from_workload(w) as sim:
        _compare(sim, w.pos_q, w.box_q, 16, 1.0, 1.0, 1.0, 3.8)


def test_evolved_flock_and_any_rule():
    """After 40 Voronoi-rule steps of the mixed workload, and on a kNN sim
    (the tissue call builds its own cells whatever the rule)."""
    w = W.voronoi_mixed(eta=0.5)
    with vk.from_workload(w) as sim:
        sim.step(40)
        pos, _, _, _ = sim.state()
        _compare(sim, pos, w.box_q, w.frac_bits, 1.0, 1.0, 1.0, 3.8)
    w2 = W.uniform_system(4000, 60.0, 16, 2, input_seed=63, rule="knn", k=7)
    with vk.from_workload(w2) as sim:
        _compare(sim, w2.pos_q, w2.box_q, 16, 1.0, 0.5, 1.0, 3.6)


def test_area_sum_and_force_sum():
    w = W.uniform_system(20000, 141.0, 16, 2, input_seed=65, rule="voronoi", k=0)
    with vk.from_workload(w) as sim:
        a, _, _, f = sim.tissue(1.0, 1.0, 1.0, 3.8)
    L = w.box_q[0] / 2.0 ** 16
    assert a.sum() == pytest.approx(L * L, rel=1e-12)
    assert np.abs(f.sum(axis=0)).max() < 1e-9 * np.abs(f).max() * np.sqrt(w.n)


def test_degenerate_inputs_are_reported():
    w = W.uniform_system(200, 14.0, 16, 2, input_seed=67, rule="voronoi", k=0)
    pos = w.pos_q.copy()
    pos[5] = pos[6]
    with vk.Sim.create(pos, w.dir, w.box_q, 16, rule="voronoi") as sim:
        with pytest.raises(vk.VKError) as e:
            sim.tissue(1.0, 1.0, 1.0, 3.8)
        assert e.value.status == vk.VK_ERR_DEGENERATE
    pos, box = W.square_lattice(8, 1 << 16, 3)
    with vk.Sim.create(pos, W.random_dirs(pos.shape[0]), box, 16, rule="voronoi") as sim:
        with pytest.raises(vk.VKError) as e:
            sim.tissue(1.0, 1.0, 1.0, 3.8)
        assert e.value.status == vk.VK_ERR_DEGENERATE


def test_cells_over_32_edges_report_capacity():
    """A particle alone in a void ringed by 60 others: its 60-edge cell is
    beyond the tissue pass's 32 edges."""
    rng = np.random.default_rng(4)
    L, F, ring_r = 1 << 16, 8, 20000.0
    ang = np.arange(60) * (2 * np.pi / 60) + rng.uniform(-1e-4, 1e-4, 60)
    rad = ring_r * (1 + rng.uniform(-3e-4, 3e-4, 60))
    c = L / 2
    ring = np.stack([c + rad * np.cos(ang), c + rad * np.sin(ang)], 1)
    outer = rng.uniform(0, L, size=(600, 2))
    outer = outer[np.hypot(outer[:, 0] - c, outer[:, 1] - c) > 1.3 * ring_r]
    pos = np.concatenate([[[c + 17, c - 31]], ring, outer]).astype(np.int64).astype(np.int32)
    with vk.Sim.create(pos, W.random_dirs(pos.shape[0]), (L, L), F, rule="voronoi") as sim:
        with pytest.raises(vk.VKError) as e:
            sim.tissue(1.0, 1.0, 1.0, 3.8)
        assert e.value.status == vk.VK_ERR_CAPACITY


def test_repeated_calls_and_steps_between_them():
    """The scratch is kept between calls, and a Voronoi sim seeds the cells
    with its last neighbors: every call still matches the oracle."""
    w = W.uniform_system(2500, 50.0, 16, 2, input_seed=69, rule="voronoi", k=0, v0=0.3, eta=0.4)
    with vk.from_workload(w) as sim:
        for KA, KP, A0, P0 in PARAMS:
            pos, _, _, _ = sim.state()
            _compare(sim, pos, w.box_q, 16, KA, KP, A0, P0)
            sim.step(3)
