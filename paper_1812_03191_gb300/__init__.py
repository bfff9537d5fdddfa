"""GB300-native nested-mesh dynamical-friction solver (Velasco Romero & Masset 2018).

``inputs`` holds the seeded synthetic workloads; ``binding`` (imported lazily) is
the ctypes binding of the CUDA C-ABI library ``libdfnest.so``.
"""
__all__ = ["inputs", "binding"]


def __getattr__(name):
    if name == "binding":
        from . import binding
        return binding
    raise AttributeError(name)
