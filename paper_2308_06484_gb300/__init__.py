"""GB300-native kinetic Delaunay triangulation (moving points on the plane).

The hot path lives in the CUDA library libkdt.so (C ABI in include/kdt.h); this
package holds its Python binding (``kdt``), its build script (``build``) and the
seeded synthetic workloads (``workloads``).
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "kdt", "build"]
