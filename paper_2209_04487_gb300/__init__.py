"""GB300-native coupled Maxwell-Schroedinger time step (arXiv 2209.04487).

The compute path is libms.so (CUDA, sm_103a) behind the C ABI in
include/ms.h; ``paper_2209_04487_gb300.binding`` is its ctypes binding
(importing it loads the library and fails loudly if it is missing), and
``build.build()`` compiles the library in-tree.
"""
from . import build  # noqa: F401
