"""GPU parity of the Voronoi rule (Sec. "Computational tools: Voronoi
neighbor lists"): per-particle half-plane clipping with exact predicates
against the oracle's exact Delaunay triangulation."""
import numpy as np
import pytest

import oracle
from paper_2103_10239_gb300 import vk
from paper_2103_10239_gb300 import workloads as W
from parity import check_step

pytestmark = pytest.mark.gpu


def _same(sim, pos, box):
    off, ids = sim.neighbors()
    woff, wids = oracle.voronoi(pos, box)
    assert np.array_equal(off, woff)
    assert np.array_equal(ids, wids)
    return off, ids


@pytest.mark.parametrize("seed,n,L,bits", [(1, 3, 2.0, 10), (2, 5, 3.0, 12), (3, 12, 4.0, 16),
                                           (4, 40, 7.0, 16), (5, 257, 16.0, 16), (6, 1000, 31.6, 20),
                                           (7, 2, 1.5, 8), (8, 1, 1.0, 8)])
def test_random_small_boxes(seed, n, L, bits):
    w = W.uniform_system(n, L, bits, 2, input_seed=seed, rule="voronoi", k=0, v0=0.3, eta=0.5)
    if len({tuple(p) for p in w.pos_q}) < n:
        pytest.skip("coincident draw")
    with vk.from_workload(w) as sim:
        _same(sim, w.pos_q, w.box_q)
        for _ in range(2):
            check_step(sim, w, "voronoi")


def test_square_and_hex_lattices():
    pos, box = W.square_lattice(16, 1 << 16, 5)
    d = W.random_dirs(pos.shape[0])
    with vk.Sim.create(pos, d, box, 16, rule="voronoi") as sim:
        off, _ = _same(sim, pos, box)
        assert set(np.diff(off)) == {4}
    pos, box = W.stretched_hex_lattice(20, 24, 2 * 30000, 25981)
    d = W.random_dirs(pos.shape[0])
    with vk.Sim.create(pos, d, box, 16, rule="voronoi") as sim:
        off, _ = _same(sim, pos, box)
        assert set(np.diff(off)) == {6}


def test_mixed_workload_checks_every_100_steps():
    """N=65536, half uniform / half jittered hex, Voronoi sets checked against
    the oracle every 100 steps over 1000 steps, one teacher-forced step at
    each check."""
    w = W.voronoi_mixed(eta=0.1)
    with vk.from_workload(w) as sim:
        for c in range(10):
            check_step(sim, w, "voronoi")
            sim.step(99)
        off, ids = sim.neighbors()
        assert ids.size == 6 * w.n  # Euler: E = 3N on generic input


def test_reciprocity_and_euler_after_steps():
    w = W.voronoi_mixed(eta=0.5)
    with vk.from_workload(w) as sim:
        sim.step(5)
        off, ids = sim.neighbors()
    rows = [set(ids[off[i]:off[i + 1]]) for i in range(w.n)]
    for i in range(0, w.n, 97):
        for j in rows[i]:
            assert i in rows[j]
    assert ids.size == 6 * w.n


@pytest.mark.parametrize("occ", [1.0, 2.0, 16.0])
def test_clustered_voronoi_split_cells(occ):
    """Voronoi cells in dense clusters (split coarse cells) and sparse
    background, F=16 so that L_q stays below 2^30."""
    base = W.clustered_large(n=1 << 14)
    rng = np.random.default_rng(7)
    pos = (base.pos_q.astype(np.int64) >> 4).astype(np.int32)  # F=20 -> F=16
    pos = np.unique(pos, axis=0)[rng.permutation(np.unique(pos, axis=0).shape[0])]
    box = (base.box_q[0] >> 4, base.box_q[1] >> 4)
    w = W.Workload(name="clustered_vor", dim=2, pos_q=pos, dir=W.random_dirs(pos.shape[0]), theta=None,
                   box_q=box, frac_bits=16, rule="voronoi", k=0, v0=0.3, eta=0.2)
    with vk.from_workload(w, cell_occupancy=occ) as sim:
        _same(sim, w.pos_q, w.box_q)
        check_step(sim, w, "voronoi")


def test_density_two_large_sampled():
    w = W.precision_study("voronoi", n=1 << 18)
    with vk.from_workload(w) as sim:
        pos, _, _, _ = sim.state()
        _same(sim, pos, w.box_q)


@pytest.mark.parametrize("rebuild", [0, 1])
def test_coincident_particles_share_a_site(rebuild):
    """Reading: coincident particles form one Voronoi site, are each other's
    neighbors and share the site's neighbors (the oracle applies the same
    rule to an exact triangulation of the distinct sites).  With reuse, the
    second and third steps start from seeds that hold the twins."""
    w = W.uniform_system(200, 14.0, 16, 2, input_seed=2, rule="voronoi", k=0, v0=0.3, eta=0.3)
    pos = w.pos_q.copy()
    pos[7] = pos[3]
    pos[11] = pos[3]
    pos[40] = pos[41]
    w.pos_q = pos
    with vk.from_workload(w, voronoi_rebuild=rebuild) as sim:
        off, ids = _same(sim, pos, w.box_q)
        assert 7 in ids[off[3]:off[4]] and 3 in ids[off[11]:off[12]]
        for _ in range(3):
            check_step(sim, w, "voronoi")


def test_huge_cell_takes_the_overflow_path():
    """A particle alone in a void ringed by 60 others has a 60-edge Voronoi
    cell: more than the main kernel's polygon capacity, so it is finished by
    the overflow kernel; lists and the update must still match the oracle."""
    rng = np.random.default_rng(4)
    L = 1 << 16
    F = 8
    ring_r = 20000.0
    # evenly spaced: a ring member keeps its edge while its radial offset
    # stays below 1/cos(3 deg) - 1 = 0.14 % of the radius
    ang = np.arange(60) * (2 * np.pi / 60) + rng.uniform(-1e-4, 1e-4, 60)
    rad = ring_r * (1 + rng.uniform(-3e-4, 3e-4, 60))
    c = L / 2
    ring = np.stack([c + rad * np.cos(ang), c + rad * np.sin(ang)], 1)
    outer = rng.uniform(0, L, size=(600, 2))
    outer = outer[np.hypot(outer[:, 0] - c, outer[:, 1] - c) > 1.3 * ring_r]
    pos = np.concatenate([[[c + 17, c - 31]], ring, outer]).astype(np.int64).astype(np.int32)
    w = W.Workload(name="void", dim=2, pos_q=pos, dir=W.random_dirs(pos.shape[0]), theta=None,
                   box_q=(L, L), frac_bits=F, rule="voronoi", k=0, v0=0.2, eta=0.3)
    with vk.from_workload(w) as sim:
        off, _ = _same(sim, pos, w.box_q)
        assert off[1] - off[0] == 60
        for _ in range(2):
            check_step(sim, w, "voronoi")


@pytest.mark.parametrize("occ", [2.0, 8.0])
def test_condensed_bands_with_voids(occ):
    """Dense bands and blobs separated by large empty regions, the kind of
    state a low-noise flock condenses into: cells at void edges reach far
    across the voids, and their sites must all be found."""
    rng = np.random.default_rng(11)
    L, F = 96, 16
    t = rng.uniform(0, L, 5000)
    band = np.stack([t, 0.3 * t + 20 + rng.normal(0, 1.5, t.size)], 1)
    centers = rng.uniform(0, L, (6, 2))
    blob = centers[rng.integers(0, 6, 2000)] + rng.normal(0, 1.0, (2000, 2))
    lq = L << F
    pos = np.floor(np.concatenate([band, blob]) * (1 << F)).astype(np.int64) % lq
    pos = np.unique(pos, axis=0).astype(np.int32)
    pos = pos[rng.permutation(pos.shape[0])]
    w = W.Workload(name="bands_voids", dim=2, pos_q=pos, dir=W.random_dirs(pos.shape[0]), theta=None,
                   box_q=(lq, lq), frac_bits=F, rule="voronoi", k=0, v0=0.3, eta=0.1)
    with vk.from_workload(w, cell_occupancy=occ) as sim:
        _same(sim, pos, w.box_q)
        for _ in range(2):
            check_step(sim, w, "voronoi")


@pytest.mark.parametrize("rebuild", [0, 1])
def test_blobs_across_voids_use_the_warp_path(rebuild):
    """Two dense blobs far apart: the cells on the rim of a blob reach across
    the void to the other blob, so they see hundreds of candidates and are
    finished one warp per cell; lists and the update must match the oracle."""
    rng = np.random.default_rng(12)
    L, F = 80, 16
    blob = np.concatenate([rng.normal(20, 2.0, (1500, 2)), rng.normal(60, 2.0, (1500, 2))])
    lq = L << F
    pos = np.floor(blob * (1 << F)).astype(np.int64) % lq
    pos = np.unique(pos, axis=0).astype(np.int32)
    pos = pos[rng.permutation(pos.shape[0])]
    w = W.Workload(name="blobs", dim=2, pos_q=pos, dir=W.random_dirs(pos.shape[0]), theta=None,
                   box_q=(lq, lq), frac_bits=F, rule="voronoi", k=0, v0=0.3, eta=0.2)
    with vk.from_workload(w, voronoi_rebuild=rebuild) as sim:
        sim.set_profiling(True, counters=True)
        _same(sim, pos, w.box_q)
        check_step(sim, w, "voronoi")
        assert sim.search_stats()["max_candidates"] > 384  # some cells went to the warp path
        for _ in range(2):
            check_step(sim, w, "voronoi")


def test_reuse_of_last_steps_neighbors_changes_nothing():
    """Starting each cell from last step's neighbors (the lazy re-check)
    orders the clipping work differently but must give the same cells: 150
    steps of the 65,536-particle mixed workload, at low noise so that it
    condenses into bands and voids, are bit-identical with and without reuse,
    and the lists match the oracle at the end."""
    w = W.voronoi_mixed(eta=0.1)
    out = []
    for rebuild in (0, 1):
        with vk.from_workload(w, voronoi_rebuild=rebuild) as sim:
            sim.step(150)
            p, d, _, _ = sim.state()
            out.append((p, d, sim.order_parameter(), sim.neighbors()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])
    woff, wids = oracle.voronoi(out[0][0], w.box_q)
    for k in (0, 1):
        assert np.array_equal(out[k][3][0], woff) and np.array_equal(out[k][3][1], wids)
