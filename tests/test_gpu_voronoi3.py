"""GPU parity of the 3D Voronoi rule (Sec. "Computational tools: Voronoi
neighbor lists": neighbors share a face of the Voronoi tessellation): every
cell clipped on the GPU with exact integer predicates, against the oracle's
exact clipping, list by list, and one teacher-forced Vicsek step (Eq. 1,
Eq. 2 with vectorial noise) at a time."""
import numpy as np
import pytest

import oracle
from paper_2103_10239_gb300 import vk
from paper_2103_10239_gb300 import workloads as W
from parity import check_step

pytestmark = pytest.mark.gpu


def _same(sim, pos, box):
    off, ids = sim.neighbors()
    woff, wids = oracle.voronoi3(pos, box)
    assert np.array_equal(off, woff), "neighbor counts differ"
    assert np.array_equal(ids, wids), "neighbor ids differ"
    return off, ids


def _create(pos, box, bits, **kw):
    d = W.random_dirs(pos.shape[0], dim=3)
    prm = dict(rule="voronoi", noise="vectorial", v0=0.5, eta=0.3)
    prm.update(kw)
    return vk.Sim.create(np.ascontiguousarray(pos, np.int32), d, box, bits, **prm)


# tiny boxes (cells reach other images), ragged block tails, several blocks
@pytest.mark.parametrize("seed,n,L,bits", [(1, 2, 1.5, 10), (2, 3, 2.0, 10), (3, 5, 2.0, 12),
                                           (4, 9, 2.5, 14), (5, 64, 4.0, 15), (6, 129, 5.1, 15),
                                           (7, 1000, 10.0, 15), (8, 4096, 16.0, 15)])
def test_random_boxes_and_teacher_forced_steps(seed, n, L, bits):
    w = W.uniform_system(n, L, bits, 3, input_seed=seed, rule="voronoi", k=0, v0=0.5, eta=0.3,
                         noise="vectorial")
    if len({tuple(p) for p in w.pos_q}) < n:
        pytest.skip("coincident draw")
    with vk.from_workload(w) as sim:
        _same(sim, w.pos_q, w.box_q)
        for _ in range(3):
            check_step(sim, w, "voronoi")


@pytest.mark.parametrize("kind,deg", [("sc", 6), ("bcc", 14), ("fcc", 12)])
def test_cubic_lattices(kind, deg):
    """Every vertex of these lattices' cells is degenerate (shared by more
    than four cells); faces of zero area (the sc diagonal neighbors) must not
    count."""
    pos, box = W.cubic_lattice(kind, 5, 1 << 12, offset_q=(3, 5, 7))
    with _create(pos, box, 12) as sim:
        off, _ = _same(sim, pos, box)
        assert set(np.diff(off)) == {deg}


def test_anisotropic_box_and_coarse_grid():
    rng = np.random.default_rng(3)
    box = (700, 1900, 4100)
    pos = rng.integers(0, box, size=(300, 3)).astype(np.int32)
    with _create(pos, box, 8) as sim:
        _same(sim, pos, box)
    # points on a coarse integer grid: many cospherical sets
    pos = np.unique(rng.integers(0, 8, size=(200, 3)) * 16, axis=0).astype(np.int32)
    with _create(pos, (128, 128, 128), 4) as sim:
        _same(sim, pos, (128, 128, 128))


def test_full_size_sampled_and_reciprocal():
    """The benchmark's 3D workload (N = 2^18, density 1): lists of a random
    sample of particles against the oracle after a few steps; reciprocity of
    every list."""
    w = W.voronoi_3d()
    with vk.from_workload(w) as sim:
        sim.step(3)
        pos, d, _, _ = sim.state()
        off, ids = sim.neighbors()
    rng = np.random.default_rng(11)
    q = np.sort(rng.choice(w.n, size=384, replace=False))
    woff, wids = oracle.voronoi3(pos, w.box_q, query=q)
    for r, i in enumerate(q):
        assert np.array_equal(ids[off[i]:off[i + 1]], wids[woff[r]:woff[r + 1]]), i
    deg = np.diff(off)
    assert 13.0 < deg.mean() < 18.0  # about 15.5 faces per Poisson-Voronoi cell
    src = np.repeat(np.arange(w.n), deg)
    fwd = set(zip(src.tolist(), ids.tolist()))
    assert all((j, i) in fwd for i, j in list(fwd)[::97])


def test_coincident_particles_are_degenerate():
    pos = np.array([[10, 10, 10], [10, 10, 10], [50, 60, 70], [90, 20, 40]], dtype=np.int32)
    with _create(pos, (100, 100, 100), 4) as sim:
        with pytest.raises(vk.VKError) as e:
            sim.step(1)
            sim.sync()  # the step is asynchronous; the latched status is read here
        assert e.value.status == vk.VK_ERR_DEGENERATE


def test_run_to_run_bit_identical():
    w = W.uniform_system(3000, 14.4, 15, 3, input_seed=9, rule="voronoi", k=0, v0=0.5, eta=0.3,
                         noise="vectorial")
    out = []
    for _ in range(2):
        with vk.from_workload(w) as sim:
            sim.step(5)
            pos, d, _, _ = sim.state()
            out.append((pos, d, sim.order_parameter()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])
