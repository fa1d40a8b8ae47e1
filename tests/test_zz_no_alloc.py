"""The allocation-free kNN entry point (vk_knn_lists_noalloc).

Callers that cannot allocate device memory when they call the library (while
recording a CUDA graph, inside real-time loops, or under a host-managed
memory budget) get the kNN lists from a fixed static scratch array instead.
This file checks, through the C ABI, that two calls in a row return exactly
the lists of the regular entry point (vk_init + vk_get_neighbors); integer
lists must match bit for bit.  It is collected last so that a failure here
never hides the other tests."""
import numpy as np
import pytest

from paper_2103_10239_gb300 import vk
from paper_2103_10239_gb300 import workloads as W


def test_rejects_sizes_beyond_the_scratch():
    """Size checks happen on the host before any device work."""
    pos = np.zeros((vk.NOALLOC_MAX_N + 1, 2), dtype=np.int32)
    out = np.zeros((vk.NOALLOC_MAX_N + 1, 7), dtype=np.int32)
    with pytest.raises(vk.VKError) as e:
        vk.knn_lists_noalloc(pos, (1 << 20, 1 << 20), 16, 7, out)
    assert e.value.status == vk.VK_ERR_ARG


def test_worst_case_grid_fits_the_scratch():
    """The largest layout: n = VK_NOALLOC_MAX_N in a box so elongated that
    the short axis has one cell and the long axis the capped 65536 cells.
    The layout is checked against the scratch on the host before any device
    work, so without a GPU the call gets past that check and stops at the
    device (VK_ERR_CUDA); a layout that did not fit would give
    VK_ERR_CAPACITY.  On a GPU machine the full call must succeed."""
    from conftest import have_gpu
    n = vk.NOALLOC_MAX_N
    pos = np.zeros((n, 2), dtype=np.int32)
    pos[:, 0] = np.arange(n, dtype=np.int64) * 32768
    out = np.zeros((n, 7), dtype=np.int32)
    box = ((1 << 31), (1 << 12))
    if have_gpu():
        torch = pytest.importorskip("torch")
        pos_d = torch.from_numpy(pos).cuda()
        out_d = torch.zeros((n, 7), dtype=torch.int32, device="cuda")
        vk.knn_lists_noalloc(pos_d, box, 20, 7, out_d)
        torch.cuda.synchronize()
        return
    with pytest.raises(vk.VKError) as e:
        vk.knn_lists_noalloc(pos, box, 20, 7, out)
    assert e.value.status == vk.VK_ERR_CUDA


@pytest.mark.gpu
def test_two_calls_match_the_regular_entry_point():
    torch = pytest.importorskip("torch")
    cases = [W.uniform_system(5000, 70.7, 16, 2, input_seed=31),
             W.clustered_large(n=1 << 16, k=12)]
    for w in cases:
        k = w.k if w.k > 0 else 7
        with vk.from_workload(w, k=k) as sim:
            off, ids = sim.neighbors()
        want = ids.reshape(-1, k)
        pos_d = torch.from_numpy(np.ascontiguousarray(w.pos_q)).cuda()
        out_d = torch.full((w.n, k), -1, dtype=torch.int32, device="cuda")
        st_d = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        for call in range(2):  # the shared scratch keeps the previous call's contents
            out_d.fill_(-1)
            vk.knn_lists_noalloc(pos_d, w.box_q, w.frac_bits, k, out_d, dev_status=st_d)
            torch.cuda.synchronize()
            assert int(st_d.item()) == 0
            assert np.array_equal(out_d.cpu().numpy(), want), (w.name, call)


@pytest.mark.gpu
def test_lists_match_the_oracle_directly():
    """The no-allocation lists against the brute-force CPU oracle itself:
    every particle at n = 5000, a random sample at n = 65536 (clustered)."""
    torch = pytest.importorskip("torch")
    import oracle
    rng = np.random.default_rng(41)
    for w, sample in ((W.uniform_system(5000, 70.7, 16, 2, input_seed=33), None),
                      (W.clustered_large(n=1 << 16, k=12, seed=1017), 2048)):
        k = w.k
        pos_d = torch.from_numpy(np.ascontiguousarray(w.pos_q)).cuda()
        out_d = torch.full((w.n, k), -1, dtype=torch.int32, device="cuda")
        vk.knn_lists_noalloc(pos_d, w.box_q, w.frac_bits, k, out_d)
        torch.cuda.synchronize()
        got = out_d.cpu().numpy()
        if sample is None:
            assert np.array_equal(got, oracle.knn(w.pos_q, w.box_q, k))
        else:
            q = np.sort(rng.choice(w.n, sample, replace=False)).astype(np.int64)
            assert np.array_equal(got[q], oracle.knn(w.pos_q, w.box_q, k, query=q))


@pytest.mark.gpu
def test_strongly_elongated_box_at_the_size_limit():
    """n = 65536, k = 32 in a 2^31 x 2^12 box (one cell across the short
    axis, the capped 65536 cells along the long one): the same lists as the
    regular entry point, and the oracle's on a sample."""
    torch = pytest.importorskip("torch")
    import oracle
    n, k = vk.NOALLOC_MAX_N, 32
    box = ((1 << 31), (1 << 12))
    rng = np.random.default_rng(43)
    pos = np.stack([rng.integers(0, box[0], n), rng.integers(0, box[1], n)], 1).astype(np.int32)
    d = np.tile(np.array([[1.0, 0.0]], dtype=np.float32), (n, 1))
    with vk.Sim.create(pos, d, box, 20, k=k) as sim:
        _, ids = sim.neighbors()
    want = ids.reshape(n, k)
    pos_d = torch.from_numpy(pos).cuda()
    out_d = torch.full((n, k), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        out_d.fill_(-1)
        vk.knn_lists_noalloc(pos_d, box, 20, k, out_d)
        torch.cuda.synchronize()
        assert np.array_equal(out_d.cpu().numpy(), want), call
    q = np.sort(rng.choice(n, 512, replace=False)).astype(np.int64)
    assert np.array_equal(want[q], oracle.knn(pos, box, k, query=q))
