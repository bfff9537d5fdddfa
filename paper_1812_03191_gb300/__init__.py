"""GB300-native nested-mesh dynamical-friction solver (Velasco Romero & Masset 2018).

``inputs`` holds the seeded synthetic workloads; ``binding`` is the ctypes binding
of the CUDA C-ABI library ``libdfnest.so`` (loaded on first use; it raises if the
library has not been built).
"""
from . import binding, inputs  # noqa: F401

__all__ = ["inputs", "binding"]
