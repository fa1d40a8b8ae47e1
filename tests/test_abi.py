"""The C ABI boundary: the library builds for sm_103a, loads, and exports
every entry point that include/vk.h declares.  No compute calls (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vk_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2103_10239_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2103_10239_gb300 import vk
    assert set(_declared()) == set(vk._SIGS)


def test_default_params_without_gpu():
    from paper_2103_10239_gb300 import vk
    p = vk.default_params()
    assert (p.rule, p.k, p.noise, p.sum_mode, p.seed) == (0, 7, 0, 1, 1)
    assert abs(p.v0 - 0.5) < 1e-7 and abs(p.eta - 0.3) < 1e-7


def test_argument_errors_are_reported_without_gpu():
    """Validation happens before any device work, so it can run here."""
    import numpy as np
    from paper_2103_10239_gb300 import vk
    pos = np.zeros((4, 2), dtype=np.int32)
    d = np.ones((4, 2), dtype=np.float32)
    with pytest.raises(vk.VKError) as e:
        vk.Sim.create(pos, d, (100, 100), 0, k=7)  # k >= N
    assert e.value.status == vk.VK_ERR_ARG
    with pytest.raises(vk.VKError) as e:
        vk.Sim.create(pos, d, (1 << 31, 1 << 31), 0, k=2, rule="voronoi")
    assert e.value.status == vk.VK_ERR_RANGE
    with pytest.raises(vk.VKError) as e:
        vk.Sim.create(pos, d, (1000, 1000), 30, k=2, v0=1.0)  # step of 2^30 grid units
    assert e.value.status == vk.VK_ERR_RANGE
    # 3D Voronoi: exact predicates in int128 need box edges <= 2^23
    p3 = np.zeros((4, 3), dtype=np.int32)
    d3 = np.ones((4, 3), dtype=np.float32)
    with pytest.raises(vk.VKError) as e:
        vk.Sim.create(p3, d3, (1 << 23, (1 << 23) + 1, 1 << 23), 16, rule="voronoi", noise="vectorial")
    assert e.value.status == vk.VK_ERR_RANGE
    with pytest.raises(vk.VKError) as e:
        vk.Sim.create(p3, d3, (1000, 1000, 1000), 8, rule="voronoi")  # 3D needs vectorial noise
    assert e.value.status == vk.VK_ERR_ARG


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2103_10239_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "vk_oracle" not in txt, f


def test_rule_variant_argument_errors_without_gpu():
    """The metric radius and the field of view are validated on the host."""
    import numpy as np
    from paper_2103_10239_gb300 import vk
    pos = np.zeros((4, 2), dtype=np.int32)
    d = np.ones((4, 2), dtype=np.float32)
    p3 = np.zeros((4, 3), dtype=np.int32)
    d3 = np.ones((4, 3), dtype=np.float32)
    bad = [
        (dict(rule="metric", r0=-1.0), vk.VK_ERR_ARG),
        (dict(rule="metric", r0=float("inf")), vk.VK_ERR_ARG),
        (dict(k=2, fov=1, fov_cos=1.5), vk.VK_ERR_ARG),
        (dict(k=2, fov=1, fov_cos=float("nan")), vk.VK_ERR_ARG),
        (dict(k=2, fov=2), vk.VK_ERR_ARG),
        (dict(rule="voronoi", fov=1, fov_cos=0.0), vk.VK_ERR_ARG),
        (dict(rule="metric", r0=1e6), vk.VK_ERR_RANGE),  # r0 * 2^16 above 2^31
        (dict(rule="voronoi", voronoi3_kernel=2), vk.VK_ERR_ARG),
    ]
    for kw, status in bad:
        with pytest.raises(vk.VKError) as e:
            vk.Sim.create(pos, d, (100, 100), 16, **kw)
        assert e.value.status == status, kw
    with pytest.raises(vk.VKError) as e:
        vk.Sim.create(p3, d3, (100, 100, 100), 16, k=2, noise="vectorial", fov=1, fov_cos=0.0)
    assert e.value.status == vk.VK_ERR_ARG


def test_rule_variant_defaults():
    from paper_2103_10239_gb300 import vk
    p = vk.default_params()
    assert (p.fov, p.r0, p.fov_cos) == (0, 1.0, -1.0)
    assert vk.default_params(rule="metric").rule == vk.VK_RULE_METRIC
    assert vk.default_params().voronoi3_kernel == 0  # one thread per 3D Voronoi cell


def test_tissue_argument_errors_without_gpu():
    """Host-side checks of vk_get_tissue come before any device work."""
    from paper_2103_10239_gb300 import vk
    lib = vk.load()
    assert lib.vk_get_tissue(None, 0, 1.0, 1.0, 1.0, 3.8, None, None, None, None) == vk.VK_ERR_ARG
