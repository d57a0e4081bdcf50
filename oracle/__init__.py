"""ctypes wrapper of the FP64 CPU oracle (hweno_oracle.c).

TEST INFRASTRUCTURE ONLY: this package is the oracle of the CUDA path.  Only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline / reference legs import it; the
product package (paper_2402_03074_gb300) never does, and this package never imports the
product.  It follows the paper (arXiv 2402.03074) step by step; see hweno_oracle.c for the
equations each function states and the readings taken where the paper is garbled.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hweno_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ADVECTION, BURGERS, EULER = 0, 1, 2
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE = 0, 1, 2
W_SCALE_INVARIANT, W_ORIGINAL, W_LINEAR = 0, 1, 2
RK_MODIFIED, RK_PLAIN = 0, 1


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def _compile(target: str, openmp: bool) -> None:
    tmp = target + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           *(["-fopenmp"] if openmp else []), "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, target)


def _current(target: str) -> bool:
    return (os.path.exists(target) and os.path.getmtime(target) >= os.path.getmtime(_SRC)
            and os.path.getmtime(target) >= os.path.getmtime(os.path.join(_HERE, "hweno_oracle.h")))


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP contraction off: plain IEEE binary64 rounding), and
    liboracle_omp.so, the same source with its per-cell stage loops shared by OpenMP threads
    (when the compiler has OpenMP; otherwise that library is the serial one)."""
    if force or not _current(_LIB):
        _compile(_LIB, False)
    if force or not _current(_LIB_OMP):
        try:
            _compile(_LIB_OMP, True)
        except subprocess.CalledProcessError:
            _compile(_LIB_OMP, False)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("eq", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double),
        ("y1", ctypes.c_double), ("ax", ctypes.c_double), ("ay", ctypes.c_double),
        ("gam", ctypes.c_double), ("bc", ctypes.c_int * 4), ("characteristic", ctypes.c_int),
        ("weights", ctypes.c_int), ("rk", ctypes.c_int), ("gamma_lo", ctypes.c_double),
        ("eps", ctypes.c_double), ("cfl", ctypes.c_double),
    ]


_lib = None
_lib_omp = None


def lib(threads: int = 0):
    """The serial oracle (threads = 0), or the OpenMP build set to `threads` threads."""
    global _lib, _lib_omp
    if threads > 0:
        if _lib_omp is None:
            build()
            _lib_omp = _declare(ctypes.CDLL(_LIB_OMP))
        _lib_omp.orc_set_threads(threads)
        return _lib_omp
    if _lib is None:
        build()
        _lib = _declare(ctypes.CDLL(_LIB))
    return _lib


def threads_available(threads: int) -> int:
    """Threads the OpenMP build will use when asked for `threads` (1 without OpenMP)."""
    return lib(threads).orc_set_threads(threads)


def _declare(L):
    """Argument and result types of the oracle's C functions."""
    P = ctypes.POINTER(_Problem)
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.orc_recon1d.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
    L.orc_recon1d.restype = None
    L.orc_recon2d.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
    L.orc_recon2d.restype = None
    L.orc_eigen.argtypes = [P, dp, ctypes.c_int, dp, dp]
    L.orc_eigen.restype = ctypes.c_int
    L.orc_alpha.argtypes = [P, dp, dp]
    L.orc_alpha.restype = None
    L.orc_stage.argtypes = [P, ctypes.c_int, dp, dp, dp, dp, ctypes.c_double, dp]
    L.orc_stage.restype = ctypes.c_int
    L.orc_stage_cells.argtypes = [P, ctypes.c_int, dp, dp, dp, dp, ctypes.c_double,
                                  ctypes.c_int64, i64p, dp, dp]
    L.orc_stage_cells.restype = ctypes.c_int
    L.orc_step.argtypes = [P, dp, dp, ctypes.c_double, ctypes.c_double, dp]
    L.orc_step.restype = ctypes.c_int
    L.orc_run.argtypes = [P, dp, dp, ctypes.c_double, ctypes.c_int64, ctypes.c_double, i64p]
    L.orc_run.restype = ctypes.c_int
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_set_threads.restype = ctypes.c_int
    return L


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Problem:
    """The oracle's own statement of a problem u_t + f(u)_x (+ g(u)_y) = 0 (Sec. 2)."""
    dim: int = 1
    eq: int = ADVECTION
    nx: int = 16
    ny: int = 1
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    ax: float = 1.0
    ay: float = 1.0
    gam: float = 1.4
    bc: tuple = (BC_PERIODIC,) * 4
    characteristic: int = 1
    weights: int = W_SCALE_INVARIANT
    rk: int = RK_MODIFIED
    gamma_lo: float = 1.0 / 400.0
    eps: float = 1e-10
    cfl: float = 0.6

    @property
    def ncomp(self) -> int:
        if self.eq == EULER:
            return 3 if self.dim == 1 else 4
        return 1

    @property
    def nmom(self) -> int:
        return 2 if self.dim == 1 else 3

    @property
    def shape(self):
        return (self.ncomp, self.nmom, self.ny, self.nx)

    def c(self) -> _Problem:
        p = _Problem()
        for name, _ in _Problem._fields_:
            if name == "bc":
                p.bc = (ctypes.c_int * 4)(*self.bc)
            else:
                setattr(p, name, getattr(self, name))
        return p


def recon1d(ub, vb, weights=W_SCALE_INVARIANT, gamma_lo=1.0 / 400.0, eps=1e-10) -> dict:
    """Steps 1-3 of Sec. 2.1 on one stencil; returns every intermediate quantity."""
    ub = np.ascontiguousarray(ub, dtype=np.float64)
    vb = np.ascontiguousarray(vb, dtype=np.float64)
    out = np.zeros(27)
    lib().orc_recon1d(_dp(ub), _dp(vb), weights, gamma_lo, eps, _dp(out))
    return dict(c0=out[0:5], c1=out[5:7], c2=out[7:9], beta=out[9:12], tau=out[12],
                uave=out[13], omega=out[14:17], C=out[17:22], pts=out[22:26], vhat=out[26])


def recon2d(ub, vb, wb, weights=W_SCALE_INVARIANT, gamma_lo=1.0 / 400.0, eps=1e-10) -> dict:
    """Steps 1-3 of Sec. 2.2 on one 3x3 stencil; returns every intermediate quantity."""
    ub = np.ascontiguousarray(ub, dtype=np.float64)
    vb = np.ascontiguousarray(vb, dtype=np.float64)
    wb = np.ascontiguousarray(wb, dtype=np.float64)
    out = np.zeros(62)
    lib().orc_recon2d(_dp(ub), _dp(vb), _dp(wb), weights, gamma_lo, eps, _dp(out))
    return dict(c0=out[0:15], cm=out[15:27].reshape(4, 3), beta=out[27:32], tau=out[32],
                uave=out[33], omega=out[34:39], pts=out[39:60], vhat=out[60], what=out[61])


def eigen(prob: Problem, ubar, direction=0):
    n = prob.ncomp
    ub = np.ascontiguousarray(ubar, dtype=np.float64)
    R = np.zeros(n * n)
    L = np.zeros(n * n)
    pc = prob.c()
    rc = lib().orc_eigen(ctypes.byref(pc), _dp(ub), direction, _dp(R), _dp(L))
    if rc != 0:
        raise ValueError("non-physical state")
    return R.reshape(n, n), L.reshape(n, n)


def alpha(prob: Problem, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == prob.shape
    a = np.zeros(2)
    pc = prob.c()
    lib().orc_alpha(ctypes.byref(pc), _dp(U), _dp(a))
    return a


def stage(prob: Problem, k: int, Uin, Un, Vh, alpha_in, dt, threads: int = 0):
    """One stage of Eq. 2.13; returns (Uout, Vh, status). Vh is filled when k == 1.
    threads > 0: the OpenMP build with that many threads (bitwise the same result)."""
    Uin = np.ascontiguousarray(Uin, dtype=np.float64)
    Un = np.ascontiguousarray(Un, dtype=np.float64)
    if Vh is None:
        Vh = np.zeros((prob.ncomp, prob.nmom - 1, prob.ny, prob.nx))
    Vh = np.ascontiguousarray(Vh, dtype=np.float64).copy()
    Uout = np.zeros(prob.shape)
    a = np.ascontiguousarray(alpha_in, dtype=np.float64)
    pc = prob.c()
    st = lib(threads).orc_stage(ctypes.byref(pc), k, _dp(Uin), _dp(Un), _dp(Vh), _dp(a), dt,
                                _dp(Uout))
    return Uout, Vh, st


def stage_cells(prob: Problem, k: int, Uin, Un, Vh, alpha_in, dt, cells):
    """The stage evaluated at the listed flat cell indices: (out[ncell, NC, NM], vh, status)."""
    Uin = np.ascontiguousarray(Uin, dtype=np.float64)
    Un = np.ascontiguousarray(Un, dtype=np.float64)
    if Vh is None:
        Vh = np.zeros((prob.ncomp, prob.nmom - 1, prob.ny, prob.nx))
    Vh = np.ascontiguousarray(Vh, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros((len(cells), prob.ncomp, prob.nmom))
    vho = np.zeros((len(cells), prob.ncomp, prob.nmom - 1))
    a = np.ascontiguousarray(alpha_in, dtype=np.float64)
    pc = prob.c()
    st = lib().orc_stage_cells(ctypes.byref(pc), k, _dp(Uin), _dp(Un), _dp(Vh), _dp(a), dt,
                               len(cells), cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               _dp(out), _dp(vho))
    return out, vho, st


def step(prob: Problem, U, t=0.0, t_end=float("inf"), dt_fixed=0.0, threads: int = 0):
    """One time step (in a copy); returns (U, t, dt, status)."""
    U = np.ascontiguousarray(U, dtype=np.float64).copy()
    tt = ctypes.c_double(t)
    dt = ctypes.c_double(0.0)
    pc = prob.c()
    st = lib(threads).orc_step(ctypes.byref(pc), _dp(U), ctypes.byref(tt), t_end, dt_fixed,
                               ctypes.byref(dt))
    return U, tt.value, dt.value, st


def run(prob: Problem, U, t=0.0, t_end=float("inf"), max_steps=-1, dt_fixed=0.0,
        threads: int = 0):
    """Steps until t_end or max_steps; returns (U, t, steps, status).  threads > 0: the
    OpenMP build with that many threads (bitwise the same result as the serial one)."""
    U = np.ascontiguousarray(U, dtype=np.float64).copy()
    tt = ctypes.c_double(t)
    ns = ctypes.c_int64(0)
    pc = prob.c()
    st = lib(threads).orc_run(ctypes.byref(pc), _dp(U), ctypes.byref(tt), t_end, max_steps,
                              dt_fixed, ctypes.byref(ns))
    return U, tt.value, ns.value, st


# ------------------------------------------------------------------------------------------
# floating-point operation count of one stage (flop_count.cpp: the oracle's source compiled
# with a counting scalar)
# ------------------------------------------------------------------------------------------
_FLOP_SRC = os.path.join(_HERE, "flop_count.cpp")
_FLOP_LIB = os.path.join(_HERE, "libflopcount.so")
_flop = None


def build_flop_count(force: bool = False) -> str:
    deps = (_FLOP_SRC, _SRC, os.path.join(_HERE, "hweno_oracle.h"))
    if (not force and os.path.exists(_FLOP_LIB)
            and all(os.path.getmtime(_FLOP_LIB) >= os.path.getmtime(d) for d in deps)):
        return _FLOP_LIB
    tmp = _FLOP_LIB + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                    tmp, _FLOP_SRC], check=True, cwd=_HERE)
    os.replace(tmp, _FLOP_LIB)
    return _FLOP_LIB


FLOP_KINDS = ("add", "sub", "mul", "div", "sqrt", "total")


def count_stage_flops(prob: Problem, k: int, Uin, Un=None, Vh=None, alpha_in=None, dt=1e-3):
    """Floating-point operations of one oracle stage on the given data.  Returns a dict:
    'dataflow' -- the distinct data-dependent operations (add, sub, mul, div, sqrt, total)
    on which a stage output depends, after merging repeated identical operations and the
    identities x*1, x*0, x+0, x-0, x/1; 'executed' -- every data-dependent operation the
    oracle executes; 'wave_speeds' -- the executed operations of the LF speeds of all cells
    of the output (the next stage's alpha).  Comparisons, negations and |x| are not counted."""
    global _flop
    if _flop is None:
        build_flop_count()
        L = ctypes.CDLL(_FLOP_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_count_stage_flops.argtypes = [ctypes.POINTER(_Problem), ctypes.c_int, dp, dp, dp,
                                            dp, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]
        L.orc_count_stage_flops.restype = ctypes.c_int
        _flop = L
    Uin = np.ascontiguousarray(Uin, dtype=np.float64)
    Un = Uin if Un is None else np.ascontiguousarray(Un, dtype=np.float64)
    if Vh is None:
        Vh = np.zeros((prob.ncomp, prob.nmom - 1, prob.ny, prob.nx))
    Vh = np.ascontiguousarray(Vh, dtype=np.float64)
    a = alpha(prob, Uin) if alpha_in is None else np.ascontiguousarray(alpha_in, dtype=np.float64)
    counts = (ctypes.c_int64 * 18)()
    pc = prob.c()
    st = _flop.orc_count_stage_flops(ctypes.byref(pc), k, _dp(Uin), _dp(Un), _dp(Vh), _dp(a), dt,
                                     counts)
    c = list(counts)
    return {"dataflow": dict(zip(FLOP_KINDS, c[0:6])), "executed": dict(zip(FLOP_KINDS, c[6:12])),
            "wave_speeds": dict(zip(FLOP_KINDS, c[12:18])), "status": st}
