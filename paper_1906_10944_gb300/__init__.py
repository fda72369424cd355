"""GB300-native GenEO two-level overlapping Schwarz hot path.

The compute path is libgeneo.so (CUDA for sm_103a, C ABI in include/geneo.h);
``geneo`` is its ctypes binding and ``build`` compiles it in-tree.
"""
from . import geneo  # noqa: F401
