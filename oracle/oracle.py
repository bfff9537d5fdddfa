"""ctypes wrapper of the plain-C FP64 oracle (``dfnest_oracle.c``).

Test infrastructure only (see the package docstring).  ``build_oracle()`` compiles
the C file with ``gcc -O2 -ffp-contract=off`` next to this module;
``build_oracle(omp=True)`` compiles the same file with ``-fopenmp`` as well, a build
that runs the oracle's plane loops on several host cores with the same results (it
exists to time the oracle on all cores).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dfnest_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}


class BC:
    PERIODIC = 0
    OUTFLOW = 1
    INFLOW = 2
    REFLECT = 3


class OracleParams(C.Structure):
    _fields_ = [
        ("gamma", C.c_double),
        ("rho0", C.c_double),
        ("cs", C.c_double),
        ("mach", C.c_double),
        ("flow_dir", C.c_double * 3),
        ("GM", C.c_double),
        ("eps", C.c_double),
        ("chi", C.c_double),
        ("L", C.c_double),
        ("lum_sigma", C.c_double),
        ("cfl", C.c_double),
        ("cfl_diff", C.c_double),
        ("dt_fixed", C.c_double),
        ("xi_mode", C.c_int),
        ("bc", C.c_int * 6),
        ("diff_face_rho", C.c_int),
        ("hydro_on", C.c_int),
        ("band", C.c_int),
        ("av_c2", C.c_double),
    ]


def build_oracle(force: bool = False, omp: bool = False) -> str:
    """Compile liboracle.so (plain C, FP64, no fused multiply-add), or with omp the
    OpenMP build liboracle_omp.so of the same file."""
    out = _LIB_OMP if omp else _LIB
    with _lock:
        if force or not os.path.exists(out) or os.path.getmtime(out) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "dfnest_oracle.h"))
        ):
            tmp = out + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared"]
                + (["-fopenmp"] if omp else []) + ["-o", tmp, _SRC, "-lm"]
            )
            os.replace(tmp, out)
    return out


def _load(omp: bool = False):
    if omp not in _libs:
        lib = C.CDLL(build_oracle(omp=omp))
        P = C.POINTER
        dp = P(C.c_double)
        lib.or_create.restype = C.c_void_p
        lib.or_create.argtypes = [C.c_int, P(C.c_int), dp, dp, C.c_int, P(OracleParams)]
        lib.or_create_ground.restype = C.c_void_p
        lib.or_create_ground.argtypes = [C.c_int, P(C.c_int), P(C.c_int), dp, dp, C.c_int,
                                         P(OracleParams)]
        lib.or_destroy.argtypes = [C.c_void_p]
        lib.or_step.argtypes = [C.c_void_p, C.c_int]
        lib.or_compute_dt.restype = C.c_double
        lib.or_compute_dt.argtypes = [C.c_void_p, dp]
        lib.or_time.restype = C.c_double
        lib.or_time.argtypes = [C.c_void_p]
        lib.or_last_dt.restype = C.c_double
        lib.or_last_dt.argtypes = [C.c_void_p]
        lib.or_force.argtypes = [C.c_void_p, dp]
        for nm in ("or_get_field", "or_get_full"):
            getattr(lib, nm).restype = C.c_int
            getattr(lib, nm).argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
        for nm in ("or_set_field", "or_set_full"):
            getattr(lib, nm).restype = C.c_int
            getattr(lib, nm).argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
        lib.or_commup.argtypes = [C.c_void_p, C.c_int]
        lib.or_commmean.argtypes = [C.c_void_p, C.c_int]
        lib.or_fill_bc.argtypes = [C.c_void_p]
        lib.or_xi_search.restype = C.c_double
        lib.or_xi_search.argtypes = [C.c_int, dp, dp, P(C.c_int)]
        lib.or_threads.restype = C.c_int
        lib.or_threads.argtypes = [C.c_int]
        _libs[omp] = lib
    return _libs[omp]


def threads(n: int = 0) -> int:
    """Threads of the OpenMP build (n > 0 sets them first)."""
    return _load(omp=True).or_threads(int(n))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def xi_search(dt_level, cost):
    """Eq. 55-56 brute force: (best dt/C, xi word)."""
    lib = _load()
    n = len(dt_level)
    dtl = np.ascontiguousarray(dt_level, dtype=np.float64)
    cst = np.ascontiguousarray(cost, dtype=np.float64)
    xi = (C.c_int * max(n - 1, 1))()
    r = lib.or_xi_search(n, _dp(dtl), _dp(cst), xi)
    return r, [xi[i] for i in range(n - 1)]


class Oracle:
    """One nested hierarchy advanced by the FP64 oracle."""

    def __init__(self, n_levels, n, lo, hi, G, params: dict, n0=None, omp=False):
        """n: cells per axis of every level; n0 (optional): of the ground level only;
        omp: run on the OpenMP build (same results, several host cores)"""
        lib = _load(omp)
        self.lib = lib
        if isinstance(n, int):
            n = (n, n, n)
        self.n = tuple(int(x) for x in n)
        if isinstance(n0, int):
            n0 = (n0, n0, n0)
        self.n0 = self.n if n0 is None else tuple(int(x) for x in n0)
        self.n_levels = int(n_levels)
        self.G = int(G)
        p = OracleParams()
        for k, v in params.items():
            if k in ("flow_dir", "bc"):
                arr = getattr(p, k)
                for i, x in enumerate(v):
                    arr[i] = x
            else:
                setattr(p, k, v)
        self.params = p
        na = (C.c_int * 3)(*self.n)
        lo_ = (C.c_double * 3)(*lo)
        hi_ = (C.c_double * 3)(*hi)
        n0_ = (C.c_int * 3)(*self.n0)
        self.h = lib.or_create_ground(self.n_levels, n0_, na, lo_, hi_, self.G, C.byref(p))
        if not self.h:
            raise ValueError("oracle rejected the hierarchy (sizes, offsets or ghost width)")

    def close(self):
        if self.h:
            self.lib.or_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        self.lib.or_step(self.h, int(n))

    def compute_dt(self):
        out = np.zeros(self.n_levels)
        dt = self.lib.or_compute_dt(self.h, _dp(out))
        return dt, out

    @property
    def t(self):
        return self.lib.or_time(self.h)

    @property
    def last_dt(self):
        return self.lib.or_last_dt(self.h)

    def force(self):
        F = np.zeros(3)
        self.lib.or_force(self.h, _dp(F))
        return F

    def level_n(self, level):
        return self.n0 if level == 0 else self.n

    def get_field(self, level, field):
        nx, ny, nz = self.level_n(level)
        out = np.zeros(nx * ny * nz)
        if self.lib.or_get_field(self.h, level, field, _dp(out)):
            raise IndexError
        return out.reshape(nz, ny, nx)

    def set_field(self, level, field, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).ravel()
        m = self.level_n(level)
        assert a.size == m[0] * m[1] * m[2]
        if self.lib.or_set_field(self.h, level, field, _dp(a)):
            raise IndexError

    def full_shape(self, level=0):
        return tuple(x + 2 * self.G for x in self.level_n(level)[::-1])

    def get_full(self, level, field):
        out = np.zeros(int(np.prod(self.full_shape(level))))
        if self.lib.or_get_full(self.h, level, field, _dp(out)):
            raise IndexError
        return out.reshape(self.full_shape(level))

    def set_full(self, level, field, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).ravel()
        if self.lib.or_set_full(self.h, level, field, _dp(a)):
            raise IndexError

    def commup(self, coarse_level):
        self.lib.or_commup(self.h, coarse_level)

    def commmean(self, coarse_level):
        self.lib.or_commmean(self.h, coarse_level)

    def fill_bc(self):
        self.lib.or_fill_bc(self.h)
