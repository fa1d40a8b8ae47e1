"""Pins for the oracle's k-nearest-neighbor rule.

The rule (Sec. "Metric and topological flocking models"): each particle
interacts with its k nearest others, at any distance, in a periodic box.
Readings: squared minimum-image distance in exact integers, order (D, id),
self excluded.  Pins: an independent Python brute force, textbook lattice
shells (including the id tie-break), scipy's periodic k-d tree on tie-free
inputs, and the symmetries of the definition.
"""
import numpy as np
import pytest

from oracle import brute
from paper_2103_10239_gb300 import workloads as W


@pytest.mark.parametrize("seed,n,dim,k,bits", [
    (1, 40, 2, 7, 12), (2, 25, 2, 12, 10), (3, 60, 3, 7, 12), (4, 9, 2, 8, 6),
    (5, 50, 2, 6, 3),   # 3-bit grid: many exact distance ties
    (6, 30, 3, 7, 3),
])
def test_knn_matches_python_brute_force(orc, seed, n, dim, k, bits):
    rng = np.random.default_rng(seed)
    box = tuple(int(b) for b in rng.integers(1 << (bits - 1), 1 << bits, size=dim))
    pos = np.stack([rng.integers(0, b, size=n) for b in box], axis=1).astype(np.int32)
    got = orc.knn(pos, box, k)
    want = np.array(brute.knn_brute(pos, box, k))
    assert np.array_equal(got, want)


def _lattice_shell_ids(m, a, i, shell_d2):
    pos, box = W.square_lattice(m, a)
    L = box[0]
    d = pos.astype(np.int64) - pos[i]
    d = np.where(2 * d > L, d - L, d)
    d = np.where(2 * d <= -L, d + L, d)
    D = (d * d).sum(1)
    return sorted(int(j) for j in np.nonzero(D == shell_d2 * a * a)[0])


@pytest.mark.parametrize("m,a", [(6, 1 << 16), (9, 1000), (4, 3)])
def test_square_lattice_shells(orc, m, a):
    """First shell: 4 sites at distance a; second: 4 at a*sqrt(2)."""
    pos, box = W.square_lattice(m, a)
    n = pos.shape[0]
    k4 = orc.knn(pos, box, 4)
    k8 = orc.knn(pos, box, 8)
    k7 = orc.knn(pos, box, 7)
    for i in range(n):
        s1 = _lattice_shell_ids(m, a, i, 1)
        s2 = _lattice_shell_ids(m, a, i, 2)
        assert len(s1) == 4 and len(s2) == 4
        assert list(k4[i]) == s1           # ties broken by id
        assert list(k8[i]) == s1 + s2
        assert list(k7[i]) == s1 + s2[:3]  # the 3 lowest ids of shell 2


def test_min_image_half_box(orc):
    """Distance exactly L/2 is the same through either image; ordering then
    falls back to the id."""
    L = 1000
    pos = np.array([[0, 0], [500, 0], [0, 500], [250, 250]], dtype=np.int32)
    got = orc.knn(pos, (L, L), 3)
    # from particle 0: D(3)=125000 < D(1)=D(2)=250000
    assert list(got[0]) == [3, 1, 2]


def test_knn_against_scipy_periodic_kdtree(orc):
    spatial = pytest.importorskip("scipy.spatial")
    w = W.uniform_system(3000, 50.0, 16, 2, input_seed=11)
    pos = w.pos_q.astype(np.float64)
    tree = spatial.cKDTree(pos, boxsize=np.array(w.box_q, dtype=np.float64))
    dist, idx = tree.query(pos, k=8)
    got = orc.knn(w.pos_q, w.box_q, 7)
    # tie-free input (checked): the sets and the order must agree exactly
    d2 = np.rint(dist[:, 1:] ** 2).astype(np.int64)
    assert np.all(np.diff(d2, axis=1) > 0)
    assert np.array_equal(got, idx[:, 1:])


def test_knn_3d_against_scipy(orc):
    spatial = pytest.importorskip("scipy.spatial")
    w = W.uniform_system(2000, 2000 ** (1 / 3), 12, 3, input_seed=12)
    tree = spatial.cKDTree(w.pos_q.astype(np.float64), boxsize=np.array(w.box_q, dtype=np.float64))
    dist, idx = tree.query(w.pos_q.astype(np.float64), k=8)
    got = orc.knn(w.pos_q, w.box_q, 7)
    d2 = np.rint(dist[:, 1:] ** 2).astype(np.int64)
    tie_free = np.all(np.diff(d2, axis=1) > 0, axis=1)
    assert tie_free.mean() > 0.9
    assert np.array_equal(got[tie_free], idx[tie_free, 1:])


def test_translation_invariance(orc):
    w = W.uniform_system(500, 20.0, 10, 2, input_seed=13)
    base = orc.knn(w.pos_q, w.box_q, 7)
    for shift in [(1, 0), (w.box_q[0] // 2, 3), (w.box_q[0] - 1, w.box_q[1] - 7)]:
        moved = np.mod(w.pos_q.astype(np.int64) + np.array(shift), np.array(w.box_q)).astype(np.int32)
        assert np.array_equal(orc.knn(moved, w.box_q, 7), base)


def test_relabel_permutes_lists(orc):
    w = W.uniform_system(400, 20.0, 16, 2, input_seed=14)
    base = orc.knn(w.pos_q, w.box_q, 7)
    perm = np.random.default_rng(3).permutation(w.n)
    inv = np.argsort(perm)
    got = orc.knn(w.pos_q[perm], w.box_q, 7)
    # particle perm[a] is now labelled a; its neighbor j is labelled inv[j]
    assert np.array_equal(got, inv[base[perm]])


def test_non_reciprocity_in_clustered_input(orc):
    """kNN need not be reciprocal; density contrast makes that common."""
    w = W.clustered_large(n=4096)
    nb = orc.knn(w.pos_q, w.box_q, 7)
    sets = [set(r) for r in nb]
    nonrec = sum(1 for i in range(w.n) for j in nb[i] if i not in sets[j])
    assert nonrec > 0


def test_sampled_query_equals_full(orc):
    w = W.uniform_system(800, 28.0, 16, 2, input_seed=15)
    full = orc.knn(w.pos_q, w.box_q, 7)
    q = np.array([0, 5, 799, 400, 5], dtype=np.int64)
    assert np.array_equal(orc.knn(w.pos_q, w.box_q, 7, query=q), full[q])
