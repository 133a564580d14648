"""GB300-native (sm_103a) Contact Dynamics hot path (arXiv:1104.3516).

* :mod:`paper_1104_3516_gb300.cd` -- Python binding of the C ABI
  (``include/cd_api.h``) over the CUDA library ``_lib/libcd_gb300.so``.
* :mod:`paper_1104_3516_gb300.workloads` -- seeded synthetic packings.
* :func:`build` -- compiles the CUDA library and the generator in-tree.
"""
from ._build import build  # noqa: F401

__all__ = ["build"]
