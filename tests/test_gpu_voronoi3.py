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

# both kernels: one thread per cell (0) and one warp per cell (1)
KERNELS = pytest.mark.parametrize("kern", [0, 1], ids=["thread", "warp"])


def _same(sim, pos, box):
    off, ids = sim.neighbors()
    woff, wids = oracle.voronoi3(pos, box)
    assert np.array_equal(off, woff), "neighbor counts differ"
    assert np.array_equal(ids, wids), "neighbor ids differ"
    return off, ids


def _create(pos, box, bits, kern=0, **kw):
    d = W.random_dirs(pos.shape[0], dim=3)
    prm = dict(rule="voronoi", noise="vectorial", v0=0.5, eta=0.3, voronoi3_kernel=kern)
    prm.update(kw)
    return vk.Sim.create(np.ascontiguousarray(pos, np.int32), d, box, bits, **prm)


# tiny boxes (cells reach other images), ragged block tails, several blocks
@pytest.mark.parametrize("seed,n,L,bits", [(1, 2, 1.5, 10), (2, 3, 2.0, 10), (3, 5, 2.0, 12),
                                           (4, 9, 2.5, 14), (5, 64, 4.0, 15), (6, 129, 5.1, 15),
                                           (7, 1000, 10.0, 15), (8, 4096, 16.0, 15)])
@KERNELS
def test_random_boxes_and_teacher_forced_steps(seed, n, L, bits, kern):
    w = W.uniform_system(n, L, bits, 3, input_seed=seed, rule="voronoi", k=0, v0=0.5, eta=0.3,
                         noise="vectorial")
    if len({tuple(p) for p in w.pos_q}) < n:
        pytest.skip("coincident draw")
    with vk.from_workload(w, voronoi3_kernel=kern) as sim:
        _same(sim, w.pos_q, w.box_q)
        for _ in range(3):
            check_step(sim, w, "voronoi")


@pytest.mark.parametrize("kind,deg", [("sc", 6), ("bcc", 14), ("fcc", 12)])
@KERNELS
def test_cubic_lattices(kind, deg, kern):
    """Every vertex of these lattices' cells is degenerate (shared by more
    than four cells); faces of zero area (the sc diagonal neighbors) must not
    count."""
    pos, box = W.cubic_lattice(kind, 5, 1 << 12, offset_q=(3, 5, 7))
    with _create(pos, box, 12, kern) as sim:
        off, _ = _same(sim, pos, box)
        assert set(np.diff(off)) == {deg}
        sim.step(1)
        sim.sync()


@KERNELS
def test_anisotropic_box_and_coarse_grid(kern):
    rng = np.random.default_rng(3)
    box = (700, 1900, 4100)
    pos = rng.integers(0, box, size=(300, 3)).astype(np.int32)
    with _create(pos, box, 8, kern) as sim:
        _same(sim, pos, box)
        sim.step(1)
        sim.sync()
    # points on a coarse integer grid: many cospherical sets
    pos = np.unique(rng.integers(0, 8, size=(200, 3)) * 16, axis=0).astype(np.int32)
    with _create(pos, (128, 128, 128), 4, kern) as sim:
        _same(sim, pos, (128, 128, 128))
        sim.step(1)
        sim.sync()


@KERNELS
def test_full_size_sampled_and_reciprocal(kern):
    """The benchmark's 3D workload (N = 2^18, density 1): lists of a random
    sample of particles against the oracle after a few steps; reciprocity of
    every list."""
    w = W.voronoi_3d()
    with vk.from_workload(w, voronoi3_kernel=kern) as sim:
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


@KERNELS
def test_coincident_particles_are_degenerate(kern):
    pos = np.array([[10, 10, 10], [10, 10, 10], [50, 60, 70], [90, 20, 40]], dtype=np.int32)
    with _create(pos, (100, 100, 100), 4, kern) as sim:
        with pytest.raises(vk.VKError) as e:
            sim.step(1)
            sim.sync()  # the step is asynchronous; the latched status is read here
        assert e.value.status == vk.VK_ERR_DEGENERATE


def test_run_to_run_bit_identical_and_kernels_agree():
    """Two runs of each kernel: identical states and order parameters (the
    heading sums follow the id order, phi is summed exactly)."""
    w = W.uniform_system(3000, 14.4, 15, 3, input_seed=9, rule="voronoi", k=0, v0=0.5, eta=0.3,
                         noise="vectorial")
    out = []
    for kern in (0, 0, 1, 1):
        with vk.from_workload(w, voronoi3_kernel=kern) as sim:
            sim.step(5)
            pos, d, _, _ = sim.state()
            out.append((pos, d, sim.order_parameter()))
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0])
        assert np.array_equal(out[0][1], o[1])
        assert np.array_equal(out[0][2], o[2])


@KERNELS
def test_batched_replicas(kern):
    """Three replicas of different sizes and boxes in one sim: every
    replica's lists against the oracle after two steps."""
    ws = [W.uniform_system(n, n ** (1.0 / 3.0), 15, 3, input_seed=20 + i, rule="voronoi", k=0, v0=0.5, eta=0.3,
                           noise="vectorial") for i, n in enumerate((300, 1000, 57))]
    with vk.batch_from_workloads(ws, voronoi3_kernel=kern) as sim:
        sim.step(2)
        for r, w in enumerate(ws):
            pos = sim.state(r)[0]
            off, ids = sim.neighbors(r)
            woff, wids = oracle.voronoi3(pos, w.box_q)
            assert np.array_equal(off, woff) and np.array_equal(ids, wids), r
