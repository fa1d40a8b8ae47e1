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
