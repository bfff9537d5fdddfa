"""FP64 CPU oracle of the nested-mesh dynamical-friction solver.

Test infrastructure only: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA path (``paper_1812_03191_gb300``) and never imports it.
"""
from .oracle import Oracle, OracleParams, build_oracle, BC, threads, xi_search  # noqa: F401
