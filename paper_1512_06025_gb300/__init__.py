"""GB300-native Bernstein-Bezier DG solver for the acoustic wave system.

The compute path is libbbdg.so (hand-written sm_103a CUDA kernels behind the C ABI of
include/bbdg.h); ``bbdg`` is its thin ctypes binding and ``inputs`` the seeded synthetic
workload generators.
"""
from . import inputs  # noqa: F401
