"""GB300-native Nested Slice Sampling (arxiv 2601.23252).

The hot path -- the batched constrained-update sweep of Nested Slice Sampling --
runs in hand-written CUDA kernels for sm_103a behind the C ABI declared in
``include/nss.h`` (shared library ``libnss_gb300.so`` built in-tree).  This
package holds the thin Python binding over that ABI (``native``), the build
step (``build``) and the seeded synthetic workloads (``workloads``).

The binding is imported lazily so that the workload generators and the build
step are usable on machines without a GPU; every compute call goes through the
CUDA library and fails loudly when it is missing.
"""
from __future__ import annotations

import importlib

__all__ = ["native", "workloads", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
