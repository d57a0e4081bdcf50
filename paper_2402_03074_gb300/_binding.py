"""ctypes binding of libhweno.so: the C ABI of include/hweno.h with the same names.

Argument marshalling only: every step of the scheme runs in the library's CUDA kernels.
If the library is missing or fails to load, importing a function raises; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhweno.so")

HWENO_OK, HWENO_PENDING = 0, 1
HWENO_ERR_ARG, HWENO_ERR_OOM, HWENO_ERR_CUDA, HWENO_ERR_NONPHYSICAL = -1, -2, -3, -4
HWENO_ERR_BUSY, HWENO_ERR_TIMEOUT, HWENO_ERR_STATE = -5, -6, -7
HWENO_ADVECTION, HWENO_BURGERS, HWENO_EULER = 0, 1, 2
HWENO_BC_PERIODIC, HWENO_BC_TRANSMISSIVE, HWENO_BC_REFLECTIVE = 0, 1, 2
HWENO_FP64, HWENO_MIXED32 = 0, 1
HWENO_W_SCALE_INVARIANT, HWENO_W_ORIGINAL, HWENO_W_LINEAR = 0, 1, 2
HWENO_STATUS_NONPHYSICAL, HWENO_STATUS_DIRECT_WEIGHTS = 1, 2

_NAMES = {0: "OK", 1: "PENDING", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA",
          -4: "ERR_NONPHYSICAL", -5: "ERR_BUSY", -6: "ERR_TIMEOUT", -7: "ERR_STATE"}


class HwenoError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class hweno_problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("equation", ctypes.c_int), ("nx", ctypes.c_int),
        ("ny", ctypes.c_int), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double), ("ax", ctypes.c_double),
        ("ay", ctypes.c_double), ("gamma", ctypes.c_double), ("bc", ctypes.c_int * 4),
        ("cfl", ctypes.c_double), ("dt_fixed", ctypes.c_double), ("t_end", ctypes.c_double),
        ("precision", ctypes.c_int), ("characteristic", ctypes.c_int), ("weights", ctypes.c_int),
        ("gamma_lo", ctypes.c_double), ("eps", ctypes.c_double),
    ]


class hweno_engine_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_uint64),
                ("max_slots", ctypes.c_int), ("server_thread", ctypes.c_int)]


class hweno_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("t", ctypes.c_double), ("steps", ctypes.c_int64),
                ("t_arrive", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_finish", ctypes.c_double), ("conservation_drift", ctypes.c_double)]


def make_problem(dim=2, equation=HWENO_EULER, nx=16, ny=None, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
                 ax=1.0, ay=1.0, gamma=1.4, bc=(HWENO_BC_PERIODIC,) * 4, cfl=0.6, dt_fixed=0.0,
                 t_end=0.0, precision=HWENO_FP64, characteristic=1,
                 weights=HWENO_W_SCALE_INVARIANT, gamma_lo=1.0 / 400.0, eps=1e-10) -> hweno_problem:
    p = hweno_problem()
    p.dim, p.equation, p.nx = dim, equation, nx
    p.ny = (1 if dim == 1 else nx) if ny is None else ny
    p.x0, p.x1, p.y0, p.y1 = x0, x1, y0, y1
    p.ax, p.ay, p.gamma = ax, ay, gamma
    p.bc = (ctypes.c_int * 4)(*bc)
    p.cfl, p.dt_fixed, p.t_end = cfl, dt_fixed, t_end
    p.precision, p.characteristic, p.weights = precision, characteristic, weights
    p.gamma_lo, p.eps = gamma_lo, eps
    return p


_lib = None


def lib() -> ctypes.CDLL:
    """Load libhweno.so (raises if it is absent: there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libhweno.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(hweno_problem)
        E = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        u64 = ctypes.c_uint64
        sig = {
            "hweno_create": ([ctypes.POINTER(hweno_engine_config), ctypes.POINTER(E)], ctypes.c_int),
            "hweno_destroy": ([E], None),
            "hweno_last_error": ([E], ctypes.c_char_p),
            "hweno_engine_stream": ([E], ctypes.c_void_p),
            "hweno_ncomp": ([P], ctypes.c_int),
            "hweno_nmom": ([P], ctypes.c_int),
            "hweno_open": ([E, P, dp, ctypes.POINTER(u64)], ctypes.c_int),
            "hweno_set_state": ([E, u64, dp, ctypes.c_double], ctypes.c_int),
            "hweno_get_state": ([E, u64, dp, dp], ctypes.c_int),
            "hweno_conservation": ([E, u64, dp, dp], ctypes.c_int),
            "hweno_step": ([E, u64, dp], ctypes.c_int),
            "hweno_advance": ([E, u64, ctypes.c_double, ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
            "hweno_close": ([E, u64], ctypes.c_int),
            "hweno_submit": ([E, P, dp, ctypes.POINTER(u64)], ctypes.c_int),
            "hweno_poll": ([E, u64, dp, ctypes.POINTER(hweno_result)], ctypes.c_int),
            "hweno_serve": ([E, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "hweno_stage_device": ([P, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp],
                                   ctypes.c_int),
            "hweno_alpha_device": ([P, vp, vp, vp], ctypes.c_int),
            "hweno_autotune": ([E, P, dp, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int), dp], ctypes.c_int),
            "hweno_stage_batch_static": ([ctypes.c_int, P, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                                          vp, vp, vp], ctypes.c_int),
            "hweno_tuning_save": ([ctypes.c_char_p], ctypes.c_int),
            "hweno_tuning_load": ([ctypes.c_char_p], ctypes.c_int),
            "hweno_tuning_query": ([P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                                   ctypes.c_int),
            "hweno_fma_peak": ([ctypes.c_int, ctypes.c_int, dp], ctypes.c_int),
            "hweno_set_wait_limit": ([E, ctypes.c_double], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int, eng=None):
    if rc < 0:
        msg = lib().hweno_last_error(eng).decode() if eng else ""
        raise HwenoError(rc, msg)
    return rc


def _host(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- engine / single-solve path ------------------------------------------------------
def hweno_create(device: int = 0, hbm_budget_bytes: int = 0, max_slots: int = 0,
                 server_thread: int = 0):
    cfg = hweno_engine_config(device, hbm_budget_bytes, max_slots, server_thread)
    eng = ctypes.c_void_p()
    _check(lib().hweno_create(ctypes.byref(cfg), ctypes.byref(eng)))
    return eng


def hweno_destroy(eng) -> None:
    lib().hweno_destroy(eng)


def hweno_ncomp(p: hweno_problem) -> int:
    return lib().hweno_ncomp(ctypes.byref(p))


def hweno_nmom(p: hweno_problem) -> int:
    return lib().hweno_nmom(ctypes.byref(p))


def state_shape(p: hweno_problem):
    return (hweno_ncomp(p), hweno_nmom(p), p.ny, p.nx)


def hweno_open(eng, p: hweno_problem, U: np.ndarray) -> int:
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == state_shape(p), (U.shape, state_shape(p))
    sid = ctypes.c_uint64()
    _check(lib().hweno_open(eng, ctypes.byref(p), _host(U), ctypes.byref(sid)), eng)
    return sid.value


def hweno_set_state(eng, sid: int, U: np.ndarray, t: float = 0.0) -> None:
    U = np.ascontiguousarray(U, dtype=np.float64)
    _check(lib().hweno_set_state(eng, sid, _host(U), t), eng)


def hweno_get_state(eng, sid: int, out: np.ndarray):
    t = ctypes.c_double()
    _check(lib().hweno_get_state(eng, sid, _host(out), ctypes.byref(t)), eng)
    return out, t.value


def hweno_conservation(eng, sid: int, ncomp: int):
    """(S, A): per component the sum of the cell averages times the cell area, and the same
    sum of magnitudes, of the solve's current state."""
    S = np.zeros(ncomp)
    A = np.zeros(ncomp)
    _check(lib().hweno_conservation(eng, sid, _host(S), _host(A)), eng)
    return S, A


def hweno_step(eng, sid: int) -> float:
    dt = ctypes.c_double()
    _check(lib().hweno_step(eng, sid, ctypes.byref(dt)), eng)
    return dt.value


def hweno_advance(eng, sid: int, t_end: float, max_steps: int = -1) -> int:
    n = ctypes.c_int64()
    _check(lib().hweno_advance(eng, sid, t_end, max_steps, ctypes.byref(n)), eng)
    return n.value


def hweno_close(eng, sid: int) -> None:
    _check(lib().hweno_close(eng, sid), eng)


# ---- served path -----------------------------------------------------------------------
def hweno_submit(eng, p: hweno_problem, U: np.ndarray) -> int:
    U = np.ascontiguousarray(U, dtype=np.float64)
    tk = ctypes.c_uint64()
    _check(lib().hweno_submit(eng, ctypes.byref(p), _host(U), ctypes.byref(tk)), eng)
    return tk.value


def hweno_poll(eng, ticket: int, out: np.ndarray | None):
    info = hweno_result()
    ptr = _host(out) if out is not None else None
    rc = lib().hweno_poll(eng, ticket, ptr, ctypes.byref(info))
    if rc < 0:
        _check(rc, eng)
    return rc, info


def hweno_serve(eng, max_steps: int = 16) -> int:
    n = ctypes.c_int()
    _check(lib().hweno_serve(eng, max_steps, ctypes.byref(n)), eng)
    return n.value


# ---- device-buffer entry points (torch tensors or raw pointers) -------------------------
def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(int(x))


def hweno_stage_device(p: hweno_problem, k: int, U_in, U_n, Vh, U_out, alpha_in, alpha_out, dt,
                       status, stream=None) -> None:
    _check(lib().hweno_stage_device(ctypes.byref(p), k, _ptr(U_in), _ptr(U_n), _ptr(Vh),
                                    _ptr(U_out), _ptr(alpha_in), _ptr(alpha_out), _ptr(dt),
                                    _ptr(status), _ptr(stream)))


def hweno_alpha_device(p: hweno_problem, U, alpha_out, stream=None) -> None:
    _check(lib().hweno_alpha_device(ctypes.byref(p), _ptr(U), _ptr(alpha_out), _ptr(stream)))


def hweno_last_error(eng) -> str:
    return lib().hweno_last_error(eng).decode()


def hweno_engine_stream(eng) -> int:
    """cudaStream_t of the engine as an integer handle (for torch.cuda.ExternalStream)."""
    return lib().hweno_engine_stream(eng) or 0


# ---- launch-geometry autotuner --------------------------------------------------------
def hweno_autotune(eng, p: hweno_problem, U: np.ndarray):
    """Returns (best rows per chunk, best band count (0 = the defaults), milliseconds of one
    stage: in 2D the mean stage of the fastest three-stage sequence)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    rows = ctypes.c_int()
    bands = ctypes.c_int()
    ms = ctypes.c_double()
    _check(lib().hweno_autotune(eng, ctypes.byref(p), _host(U), ctypes.byref(rows),
                                ctypes.byref(bands), ctypes.byref(ms)), eng)
    return rows.value, bands.value, ms.value


def hweno_tuning_save(path: str) -> None:
    _check(lib().hweno_tuning_save(path.encode()))


def hweno_tuning_load(path: str) -> int:
    return _check(lib().hweno_tuning_load(path.encode()))


def hweno_tuning_query(p: hweno_problem):
    """The tuning-table entry for problem p as a dict (rows, bands, width, lanes), or None."""
    v = [ctypes.c_int() for _ in range(4)]
    rc = _check(lib().hweno_tuning_query(ctypes.byref(p), *[ctypes.byref(x) for x in v]))
    if rc == 0:
        return None
    return dict(zip(("rows", "bands", "width", "lanes"), (x.value for x in v)))


def hweno_set_wait_limit(eng, seconds: float) -> None:
    """Bound the engine's waits for the device (0: no bound); HWENO_ERR_TIMEOUT past it."""
    _check(lib().hweno_set_wait_limit(eng, seconds), eng)


def hweno_fma_peak(device: int = 0, fp64: bool = True) -> float:
    """FMA throughput of the device in flop/s (FMA = 2 flops), FP64 or FP32."""
    r = ctypes.c_double()
    _check(lib().hweno_fma_peak(device, 1 if fp64 else 0, ctypes.byref(r)))
    return r.value


HWENO_STATIC_BATCH_MAX = 16


def hweno_stage_batch_static(problems, k, U_in, U_n, Vh, U_out, alpha_in, alpha_out, dt, status,
                             stream=None) -> None:
    """One stage of several 2D solves in one launch with no device allocation (static
    scratch); the lists hold one problem / device buffer per solve."""
    n = len(problems)
    arr = (hweno_problem * max(n, 1))(*problems)

    def ptrs(xs):
        a = (ctypes.c_void_p * max(n, 1))(*[_ptr(x).value if x is not None else None for x in xs])
        return ctypes.cast(a, ctypes.c_void_p)

    _check(lib().hweno_stage_batch_static(n, arr, k, ptrs(U_in), ptrs(U_n), ptrs(Vh), ptrs(U_out),
                                          ptrs(alpha_in), ptrs(alpha_out), ptrs(dt), ptrs(status),
                                          _ptr(stream)))
