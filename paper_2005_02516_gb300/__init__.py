"""GB300-native entropy-stable DG for the 2D shallow water equations on curved
triangles (Wu, Kubatko, Chan, arXiv 2005.02516).

The compute path is libesdg.so (hand-written CUDA for sm_103a behind the C ABI
of include/esdg.h); ``esdg`` is its thin Python binding.
"""

from .esdg import Solver, load_library, EsdgError  # noqa: F401
