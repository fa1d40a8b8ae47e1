"""GB300-native non-metric (kNN / Voronoi) neighbor lists fused with the
Vicsek update (arxiv 2103.10239).

* ``paper_2103_10239_gb300.vk`` -- ctypes binding of ``libvk_nm`` (the C ABI in
  ``include/vk.h``); the library is built in-tree by ``_build.build()``.
* ``paper_2103_10239_gb300.workloads`` -- seeded synthetic inputs.

Nothing is imported eagerly so that input generation works without the
compiled library; using the binding without it raises.
"""
__all__ = ["vk", "workloads"]
