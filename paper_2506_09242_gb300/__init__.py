"""GB300-native lattice Boltzmann hot path (D3Q19 / D3Q27, two-population
fused collide-and-stream, tag-selected boundaries, FP64 reductions).

The compute runs in the CUDA library built from ``csrc/`` for sm_103a; the
Python side only marshals arguments.  Build it with ``_build.build()`` (or
``__graft_entry__.build()``).
"""
from . import lbm  # noqa: F401
from .lbm import Lattice, LBMError, UnstableError  # noqa: F401

__all__ = ["Lattice", "LBMError", "UnstableError", "lbm"]
