"""GB300-native relativistic lattice Boltzmann step (arXiv:1909.04502).

The compute path is the CUDA library ``librlbm.so`` (C ABI in
include/rlbm.h); ``rlbm`` is its thin Python binding and ``inputs`` holds the
seeded synthetic workloads.
"""
from .rlbm import Lattice, RLBMError, lib, plan  # noqa: F401
