"""GB300-native scaled-stencil P1 operators on hierarchical hybrid grids.

The compute path is libhhgs (C ABI in include/hhg.h, CUDA kernels for sm_103a in
``csrc/``); ``binding`` is its ctypes binding.  Build with ``build.build()``.
"""

from . import binding  # noqa: F401

__all__ = ["binding"]
