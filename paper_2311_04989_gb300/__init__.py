"""GB300-native GRMHD Runge-Kutta stage (arXiv:2311.04989): C-ABI CUDA library + thin binding.

``grstage`` binds ``libgrstage.so`` (built by ``build.build()``); ``inputs`` draws seeded synthetic
MeshBlocks.  There is no CPU path: every stage computation runs in the library's CUDA kernels.
"""
from . import grstage  # noqa: F401
