"""ctypes binding of libdfnest.so (C ABI in include/dfnest.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  There is no fallback: if the library is missing or no GPU is present,
the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdfnest.so")

DF_OK, DF_EINVAL, DF_ENOMEM, DF_ECUDA, DF_EUNHEALTHY, DF_ETIMEOUT, DF_EBUSY = 0, -1, -2, -3, -4, -5, -6
DF_FP64, DF_FP32_STATE = 0, 1
KERNEL_KINDS = 18

# every symbol include/dfnest.h declares
EXPORTS = (
    "df_create", "df_set_params", "df_step", "df_status", "df_force", "df_force_now",
    "df_compute_dt", "df_get_field", "df_set_field", "df_get_full", "df_set_full",
    "df_state_size", "df_get_state", "df_set_state", "df_prolong", "df_restrict",
    "df_fill_bc", "df_kernel_launches", "df_set_timing", "df_kernel_time", "df_kernel_name",
    "df_debug_full_boxes", "df_destroy", "df_xi_search", "df_last_error",
    "df_force_level_noalloc", "df_check_division",
    "df_run_bytes", "df_pool_create", "df_pool_admit", "df_pool_release", "df_pool_step",
    "df_pool_query", "df_pool_get_field", "df_pool_info", "df_pool_set_tiles",
    "df_pool_autotune", "df_pool_destroy", "df_pool_set_timing", "df_pool_kernel_time",
    "df_autotune", "df_set_tile_shapes", "df_pool_set_tile_shapes", "df_set_transport",
    "df_pool_set_transport", "df_pool_set_field", "df_create_ground", "df_run_bytes_ground",
    "df_pool_admit_ground", "df_set_allocator", "df_create_levels", "df_pool_force",
    "df_pool_history", "df_measure_fp64_peak", "df_check_df64",
)
POOL_OPS = 22
# operator order of the per-op tables (tile shapes, blocks per SM)
OP_NAMES = ("source", "compress", "frontier_diff", "diffuse", "tprep", "tflux", "tfrontier",
            "tmom", "tupdate", "vrec_source", "bc", "commup", "commmean", "zero_acc",
            "dt_level", "dt_final", "force_level", "force_final", "time", "sweep",
            "visc_q", "visc_v")
TRANSPORT_AUTO, TRANSPORT_SEPARATE, TRANSPORT_FUSED = 0, 1, 2
NOALLOC_MAX_CELLS = 4194304


# device allocator callbacks (df_set_allocator)
_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_KEEP = []  # every callback pair ever handed to the library: its owners may outlive a switch


class DfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dfnest error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [
        ("gamma", C.c_double), ("rho0", C.c_double), ("cs", C.c_double), ("mach", C.c_double),
        ("flow_dir", C.c_double * 3), ("GM", C.c_double), ("eps", C.c_double),
        ("chi", C.c_double), ("L", C.c_double), ("lum_sigma", C.c_double),
        ("cfl", C.c_double), ("cfl_diff", C.c_double), ("dt_fixed", C.c_double),
        ("xi_mode", C.c_int), ("bc", C.c_int * 6), ("diff_face_rho", C.c_int),
        ("hydro_on", C.c_int), ("band", C.c_int), ("av_c2", C.c_double),
    ]

    @classmethod
    def from_dict(cls, d: dict) -> "Params":
        p = cls()
        for k, v in d.items():
            if k in ("flow_dir", "bc"):
                arr = getattr(p, k)
                for i, x in enumerate(v):
                    arr[i] = x
            else:
                setattr(p, k, v)
        return p


_lib = None


def load(path: str = LIB_PATH):
    """Load the library (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run __graft_entry__.build() (nvcc, sm_103a)")
    lib = C.CDLL(path)
    P, dp, vp = C.POINTER, C.POINTER(C.c_double), C.c_void_p
    sig = {
        "df_create": (C.c_int, [P(vp), C.c_int, P(C.c_int), dp, dp, C.c_int, C.c_int, C.c_int, vp]),
        "df_create_ground": (C.c_int, [P(vp), C.c_int, P(C.c_int), P(C.c_int), dp, dp, C.c_int,
                                       C.c_int, C.c_int, vp]),
        "df_set_params": (C.c_int, [vp, P(Params)]),
        "df_step": (C.c_int, [vp, C.c_int, dp]),
        "df_create_levels": (C.c_int, [P(vp), C.c_int, C.c_int, dp, dp, C.c_int, C.c_int, vp,
                                       vp, vp, vp]),
        "df_pool_force": (C.c_int, [vp, C.c_int, dp, dp]),
        "df_pool_history": (C.c_int, [vp, C.c_int, C.c_int, dp, P(C.c_int)]),
        "df_measure_fp64_peak": (C.c_int, [C.c_int, C.c_int, dp, dp]),
        "df_check_df64": (C.c_int, [dp, dp, C.c_int, dp]),
        "df_status": (C.c_int, [vp, dp, dp, P(C.c_int)]),
        "df_force": (C.c_int, [vp, dp, dp]),
        "df_force_now": (C.c_int, [vp, dp]),
        "df_compute_dt": (C.c_int, [vp, dp, dp]),
        "df_get_field": (C.c_int, [vp, C.c_int, C.c_int, dp]),
        "df_set_field": (C.c_int, [vp, C.c_int, C.c_int, dp]),
        "df_get_full": (C.c_int, [vp, C.c_int, C.c_int, dp]),
        "df_set_full": (C.c_int, [vp, C.c_int, C.c_int, dp]),
        "df_state_size": (C.c_size_t, [vp]),
        "df_get_state": (C.c_int, [vp, dp, dp]),
        "df_set_state": (C.c_int, [vp, dp, C.c_double]),
        "df_prolong": (C.c_int, [vp, C.c_int]),
        "df_restrict": (C.c_int, [vp, C.c_int]),
        "df_fill_bc": (C.c_int, [vp]),
        "df_kernel_launches": (C.c_longlong, [vp]),
        "df_set_timing": (C.c_int, [vp, C.c_int]),
        "df_kernel_time": (C.c_int, [vp, C.c_int, dp, P(C.c_longlong)]),
        "df_kernel_name": (C.c_char_p, [C.c_int]),
        "df_debug_full_boxes": (C.c_int, [vp, C.c_int]),
        "df_autotune": (C.c_int, [vp, P(C.c_int)]),
        "df_set_tile_shapes": (C.c_int, [vp, P(C.c_int)]),
        "df_set_transport": (C.c_int, [vp, C.c_int]),
        "df_pool_set_transport": (C.c_int, [vp, C.c_int]),
        "df_pool_set_field": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, dp]),
        "df_pool_set_tile_shapes": (C.c_int, [vp, P(C.c_int)]),
        "df_destroy": (C.c_int, [vp]),
        "df_xi_search": (C.c_int, [C.c_int, dp, dp, P(C.c_int), dp]),
        "df_last_error": (C.c_char_p, []),
        "df_check_division": (C.c_int, [dp, dp, C.c_int, dp]),
        "df_run_bytes": (C.c_size_t, [C.c_int, P(C.c_int), C.c_int, C.c_int]),
        "df_set_allocator": (C.c_int, [vp, vp, vp]),
        "df_run_bytes_ground": (C.c_size_t, [C.c_int, P(C.c_int), P(C.c_int), C.c_int, C.c_int]),
        "df_pool_create": (C.c_int, [P(vp), C.c_size_t, C.c_int, C.c_int, vp]),
        "df_pool_admit": (C.c_int, [vp, C.c_int, P(C.c_int), dp, dp, C.c_int, P(Params),
                                    P(C.c_int)]),
        "df_pool_admit_ground": (C.c_int, [vp, C.c_int, P(C.c_int), P(C.c_int), dp, dp, C.c_int,
                                           P(Params), P(C.c_int)]),
        "df_pool_release": (C.c_int, [vp, C.c_int]),
        "df_pool_step": (C.c_int, [vp, C.c_int]),
        "df_pool_query": (C.c_int, [vp, dp, C.c_int]),
        "df_pool_get_field": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, dp]),
        "df_pool_info": (C.c_int, [vp, P(C.c_int), P(C.c_size_t), P(C.c_size_t),
                                   P(C.c_longlong)]),
        "df_pool_set_tiles": (C.c_int, [vp, P(C.c_int)]),
        "df_pool_autotune": (C.c_int, [vp, P(C.c_int)]),
        "df_pool_destroy": (C.c_int, [vp]),
        "df_pool_set_timing": (C.c_int, [vp, C.c_int]),
        "df_pool_kernel_time": (C.c_int, [vp, C.c_int, dp, P(C.c_longlong)]),
        "df_force_level_noalloc": (C.c_int, [vp, P(C.c_int), C.c_int, dp, dp, P(C.c_int),
                                             P(C.c_int), C.c_double, C.c_double, C.c_double,
                                             C.c_int, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != DF_OK:
        raise DfError(rc, _lib.df_last_error().decode())
    return rc


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def kernel_name(kind: int) -> str:
    return load().df_kernel_name(kind).decode()


def xi_search(dt_level, cost):
    lib = load()
    n = len(dt_level)
    a = np.ascontiguousarray(dt_level, dtype=np.float64)
    b = np.ascontiguousarray(cost, dtype=np.float64)
    xi = (C.c_int * max(n - 1, 1))()
    r = C.c_double()
    _check(lib.df_xi_search(n, _dp(a), _dp(b), xi, C.byref(r)))
    return r.value, [xi[i] for i in range(n - 1)]


def use_torch_allocator(on=True):
    """Contexts and pools created from now on take their device memory from PyTorch's
    caching allocator (it then shows in torch.cuda.memory_allocated and shares
    torch's cache); on=False goes back to cudaMalloc.  Owners keep the allocator
    they were created with."""
    lib = load()
    if not on:
        _check(lib.df_set_allocator(None, None, None))
        return
    import torch

    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except Exception:  # out of memory: the library reports DF_ENOMEM
            return None

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    pair = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _KEEP.append(pair)
    _check(lib.df_set_allocator(C.cast(pair[0], C.c_void_p), C.cast(pair[1], C.c_void_p), None))


def measure_fp64_peak(device=0, repeats=5):
    """(TFLOP/s, best launch ms) of the library's FP64 multiply-add probe"""
    lib = load()
    tf, ms = C.c_double(), C.c_double()
    _check(lib.df_measure_fp64_peak(int(device), int(repeats), C.byref(tf), C.byref(ms)))
    return tf.value, ms.value


def check_df64(a, b):
    """worst errors of the device's double-float conversion, sum, product and
    quotient against FP64, of the unnormalised product and quotient, the size of
    their low parts and a sum taking one of them, each in units of its bound
    (<= 1 passes)"""
    lib = load()
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    w = np.zeros(8)
    _check(lib.df_check_df64(_dp(a), _dp(b), a.size, _dp(w)))
    return w


def check_division(a, b):
    """max ulp difference of the kernels' FP64 division from IEEE division"""
    lib = load()
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    m = C.c_double()
    _check(lib.df_check_division(_dp(a), _dp(b), a.size, C.byref(m)))
    return m.value


def force_level_noalloc(rho_dev_ptr, n, G, lo, dx, child_off=None, child_n=None, GM=0.0,
                        eps=0.0, rho0=1.0, F_dev_ptr=0, stream=None, mirror=0):
    """Per-level force on device buffers, with no device allocation (see the C
    declaration).  rho_dev_ptr (the FULL density) / F_dev_ptr are device addresses
    (ints); mirror: bit d for a mirror plane at the lower face of axis d."""
    lib = load()
    ci = lambda v: (C.c_int * 3)(*v) if v is not None else None  # noqa: E731
    cd = lambda v: (C.c_double * 3)(*v)  # noqa: E731
    _check(lib.df_force_level_noalloc(C.c_void_p(rho_dev_ptr), ci(n), int(G), cd(lo), cd(dx),
                                      ci(child_off), ci(child_n), float(GM), float(eps),
                                      float(rho0), int(mirror), C.c_void_p(F_dev_ptr),
                                      C.c_void_p(stream) if stream else None))


def _shapes(shapes):
    if isinstance(shapes, int):
        flat = [shapes] * (3 * POOL_OPS)
    else:
        flat = [int(v) for row in shapes for v in row]
    if len(flat) != 3 * POOL_OPS:
        raise ValueError(f"need {POOL_OPS} x 3 tile shapes")
    return (C.c_int * (3 * POOL_OPS))(*flat)


class Sim:
    """One nested hierarchy resident on one GPU (a df_ctx)."""

    def __init__(self, n_levels, n, lo, hi, G, params: dict | None = None,
                 precision=DF_FP64, device=0, stream=None, n0=None):
        """n: cells per axis of every level; n0 (optional): of the ground level only
        (df_create_ground: n0 = 2n puts the first level over a quarter of the ground)"""
        lib = load()
        self.lib = lib
        if isinstance(n, int):
            n = (n, n, n)
        self.n = tuple(int(x) for x in n)
        if isinstance(n0, int):
            n0 = (n0, n0, n0)
        self.n0 = self.n if n0 is None else tuple(int(x) for x in n0)
        self.lo, self.hi = tuple(float(x) for x in lo), tuple(float(x) for x in hi)
        self.n_levels = int(n_levels)
        self.G = int(G)
        self.precision = precision
        h = C.c_void_p()
        na = (C.c_int * 3)(*self.n)
        n0_ = (C.c_int * 3)(*self.n0)
        lo_ = (C.c_double * 3)(*lo)
        hi_ = (C.c_double * 3)(*hi)
        st = C.c_void_p(stream) if stream else None
        _check(lib.df_create_ground(C.byref(h), self.n_levels, n0_, na, lo_, hi_, self.G,
                                    precision, device, st))
        self.h = h
        if params is not None:
            self.set_params(params)

    # lifecycle
    def close(self):
        if getattr(self, "h", None):
            self.lib.df_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # calls
    def set_params(self, params: dict):
        self.params = dict(params)
        _check(self.lib.df_set_params(self.h, C.byref(Params.from_dict(params))))

    def step(self, n=1, want_t=False):
        """advance n coarse steps (asynchronous); want_t: synchronise and return t"""
        if not want_t:
            _check(self.lib.df_step(self.h, int(n), None))
            return None
        t = C.c_double()
        _check(self.lib.df_step(self.h, int(n), C.byref(t)))
        return t.value

    def status(self):
        t, dt = C.c_double(), C.c_double()
        bad = C.c_int()
        _check(self.lib.df_status(self.h, C.byref(t), C.byref(dt), C.byref(bad)))
        return t.value, dt.value, bad.value

    @property
    def t(self):
        return self.status()[0]

    def force(self):
        F = np.zeros(3)
        along = C.c_double()
        _check(self.lib.df_force(self.h, _dp(F), C.byref(along)))
        return F, along.value

    def force_now(self):
        F = np.zeros(3)
        _check(self.lib.df_force_now(self.h, _dp(F)))
        return F

    def compute_dt(self):
        dt = C.c_double()
        lv = np.zeros(self.n_levels)
        _check(self.lib.df_compute_dt(self.h, C.byref(dt), _dp(lv)))
        return dt.value, lv

    def level_n(self, level):
        return self.n0 if level == 0 else self.n

    def get_field(self, level, field):
        nx, ny, nz = self.level_n(level)
        out = np.empty(nx * ny * nz)
        _check(self.lib.df_get_field(self.h, level, field, _dp(out)))
        return out.reshape(nz, ny, nx)

    def set_field(self, level, field, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).ravel()
        m = self.level_n(level)
        if a.size != m[0] * m[1] * m[2]:
            raise ValueError("wrong size")
        _check(self.lib.df_set_field(self.h, level, field, _dp(a)))

    def full_shape(self, level=0):
        return tuple(x + 2 * self.G for x in self.level_n(level)[::-1])

    def get_full(self, level, field):
        out = np.empty(int(np.prod(self.full_shape(level))))
        _check(self.lib.df_get_full(self.h, level, field, _dp(out)))
        return out.reshape(self.full_shape(level))

    def set_full(self, level, field, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).ravel()
        if a.size != int(np.prod(self.full_shape(level))):
            raise ValueError("wrong size")
        _check(self.lib.df_set_full(self.h, level, field, _dp(a)))

    def state_size(self):
        return int(self.lib.df_state_size(self.h))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.state_size())
        t = C.c_double()
        _check(self.lib.df_get_state(self.h, _dp(out), C.byref(t)))
        return out, t.value

    def set_state(self, state, t):
        a = np.ascontiguousarray(state, dtype=np.float64)
        _check(self.lib.df_set_state(self.h, _dp(a), float(t)))

    def prolong(self, coarse_level):
        _check(self.lib.df_prolong(self.h, coarse_level))

    def restrict(self, coarse_level):
        _check(self.lib.df_restrict(self.h, coarse_level))

    def fill_bc(self):
        _check(self.lib.df_fill_bc(self.h))

    def kernel_launches(self):
        return int(self.lib.df_kernel_launches(self.h))

    def set_timing(self, on):
        _check(self.lib.df_set_timing(self.h, 1 if on else 0))

    def kernel_time(self, kind):
        ms = C.c_double()
        n = C.c_longlong()
        _check(self.lib.df_kernel_time(self.h, kind, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def autotune(self):
        """tile shape index per (operator, direction), chosen by timing"""
        out = (C.c_int * (3 * POOL_OPS))()
        _check(self.lib.df_autotune(self.h, out))
        return [list(out[3 * o:3 * o + 3]) for o in range(POOL_OPS)]

    def set_tile_shapes(self, shapes):
        """shapes: POOL_OPS x 3 tile shape indices (or one index for all)"""
        _check(self.lib.df_set_tile_shapes(self.h, _shapes(shapes)))

    def set_transport(self, mode):
        _check(self.lib.df_set_transport(self.h, int(mode)))

    def debug_full_boxes(self, on):
        _check(self.lib.df_debug_full_boxes(self.h, 1 if on else 0))


def run_bytes(n_levels, n, G, precision=DF_FP64, n0=None):
    if isinstance(n, int):
        n = (n, n, n)
    if isinstance(n0, int):
        n0 = (n0, n0, n0)
    n0 = n if n0 is None else n0
    return int(load().df_run_bytes_ground(n_levels, (C.c_int * 3)(*n0), (C.c_int * 3)(*n), G,
                                          precision))


class Pool:
    """Many independent runs stepped together on one GPU (a df_pool)."""

    def __init__(self, budget_bytes, precision=DF_FP64, device=0, stream=None):
        lib = load()
        self.lib = lib
        self.precision = precision
        h = C.c_void_p()
        _check(lib.df_pool_create(C.byref(h), int(budget_bytes), precision, device,
                                  C.c_void_p(stream) if stream else None))
        self.h = h
        self.shapes = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.df_pool_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def admit(self, n_levels, n, lo, hi, G, params: dict, n0=None):
        """slot index, or None when the HBM budget is full; n0 as in Sim"""
        if isinstance(n, int):
            n = (n, n, n)
        if isinstance(n0, int):
            n0 = (n0, n0, n0)
        n0 = tuple(n) if n0 is None else tuple(n0)
        slot = C.c_int()
        rc = self.lib.df_pool_admit_ground(self.h, int(n_levels), (C.c_int * 3)(*n0),
                                           (C.c_int * 3)(*n), (C.c_double * 3)(*lo),
                                           (C.c_double * 3)(*hi), int(G),
                                           C.byref(Params.from_dict(params)), C.byref(slot))
        if rc == DF_EBUSY:
            return None
        _check(rc)
        self.shapes[slot.value] = (int(n_levels), tuple(n), n0)
        return slot.value

    def release(self, slot):
        _check(self.lib.df_pool_release(self.h, int(slot)))
        self.shapes.pop(slot, None)

    def step(self, n=1):
        _check(self.lib.df_pool_step(self.h, int(n)))

    def query(self, max_slots=4096):
        """array (slots, 6): F_x, F_y, F_z, t, dt, unhealthy (NaN rows for empty slots)"""
        out = np.empty(6 * max_slots)
        ns = self.lib.df_pool_query(self.h, _dp(out), max_slots)
        if ns < 0:
            _check(ns)
        return out[:6 * ns].reshape(ns, 6)

    def force(self, slot):
        """(F, t) of one slot's run after its last coarse step; raises DfError with
        DF_EUNHEALTHY when that run's state went bad"""
        F = np.zeros(3)
        t = C.c_double()
        _check(self.lib.df_pool_force(self.h, int(slot), _dp(F), C.byref(t)))
        return F, t.value

    def history(self, slot, k):
        """array (m, 4) of the last m <= k coarse steps of a slot's run, oldest first:
        F_x, F_y, F_z after the step and the time at its end"""
        out = np.empty(4 * max(int(k), 1))
        got = C.c_int()
        _check(self.lib.df_pool_history(self.h, int(slot), int(k), _dp(out), C.byref(got)))
        return out[:4 * got.value].reshape(got.value, 4)

    def set_field(self, slot, level, field, values):
        nl, n, n0 = self.shapes[slot]
        n = n0 if level == 0 else n
        a = np.ascontiguousarray(values, dtype=np.float64).reshape(-1)
        if a.size != n[0] * n[1] * n[2]:
            raise ValueError("field size does not match the run's mesh")
        _check(self.lib.df_pool_set_field(self.h, int(slot), level, field, _dp(a)))

    def get_field(self, slot, level, field):
        nl, n, n0 = self.shapes[slot]
        n = n0 if level == 0 else n
        out = np.empty(n[0] * n[1] * n[2])
        _check(self.lib.df_pool_get_field(self.h, int(slot), level, field, _dp(out)))
        return out.reshape(n[2], n[1], n[0])

    def info(self):
        a, used, budget, launches = C.c_int(), C.c_size_t(), C.c_size_t(), C.c_longlong()
        _check(self.lib.df_pool_info(self.h, C.byref(a), C.byref(used), C.byref(budget),
                                     C.byref(launches)))
        return dict(active=a.value, used=used.value, budget=budget.value,
                    launches=launches.value)

    def autotune(self):
        out = (C.c_int * POOL_OPS)()
        _check(self.lib.df_pool_autotune(self.h, out))
        return list(out)

    def set_timing(self, on):
        _check(self.lib.df_pool_set_timing(self.h, 1 if on else 0))

    def kernel_time(self, kind):
        ms = C.c_double()
        n = C.c_longlong()
        _check(self.lib.df_pool_kernel_time(self.h, kind, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def set_tile_shapes(self, shapes):
        _check(self.lib.df_pool_set_tile_shapes(self.h, _shapes(shapes)))

    def set_transport(self, mode):
        _check(self.lib.df_pool_set_transport(self.h, int(mode)))

    def set_tiles(self, blocks_per_sm):
        arr = (C.c_int * POOL_OPS)(*blocks_per_sm)
        _check(self.lib.df_pool_set_tiles(self.h, arr))
