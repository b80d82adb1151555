"""GB300 (sm_103a) random batch sum-of-Gaussians (RBSOG) force step for periodic Yukawa systems.

The compute path is librbsog (hand-written CUDA behind the C ABI in include/rbsog.h);
``rbsog`` is its ctypes binding and ``workloads`` the seeded input generators.
Importing the package does not load the library; the first binding call does, and
fails loudly when it is missing.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "rbsog", "build"]
