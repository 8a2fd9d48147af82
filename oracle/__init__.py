"""CPU oracle for time-iterated Jacobi and Gauss-Seidel stencils.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it; the library never does. It shares no
code with the CUDA path and never imports it.

``run`` calls the plain C definition in ``stencil_oracle.c`` (the naive
(d+1)-loop stencil of Section 1 / Algorithm 1, Gauss-Seidel as in Section
3.4); ``exact`` holds an independent exact-rational restatement used to pin
it. Both follow the same readings of what the paper leaves open: canonical
(lexicographic, slowest dimension first) offset order, terms summed in
descending canonical order, and the two rounding modes FMA / UNFUSED.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

STAR, BOX = 0, 1
JACOBI, GAUSS_SEIDEL = 0, 1
BC_CONSTANT, BC_PERIODIC = 0, 1
ARITH_FMA, ARITH_UNFUSED = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stencil_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, no FP contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load(path: str):
    """Load an oracle shared library from path (the default one is built by build())."""
    lib = ctypes.CDLL(path)
    lib.oracle_offsets.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.oracle_offsets.restype = ctypes.c_int
    lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    lib.oracle_run.restype = ctypes.c_int
    if hasattr(lib, "oracle_run_field"):
        lib.oracle_run_field.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        lib.oracle_run_field.restype = ctypes.c_int
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        lib = load(_LIB)
        _lib = lib
    return _lib


def offsets(dim: int, shape: int, r: int):
    """Canonical offsets as tuples of length dim (slowest component first)."""
    lib = _load()
    k = lib.oracle_offsets(dim, shape, r, None)
    if k < 0:
        raise ValueError("bad stencil")
    buf = (ctypes.c_int * (3 * k))()
    lib.oracle_offsets(dim, shape, r, buf)
    return [tuple(buf[3 * q + 3 - dim: 3 * q + 3]) for q in range(k)]


def max_threads() -> int:
    return _load().oracle_max_threads()


def run(u, T: int, *, dim: int, shape: int, r: int, weights, method: int = JACOBI,
        bc: int = BC_CONSTANT, c: float = 0.0, arith: int = ARITH_FMA, nthreads: int = 0,
        lib=None, field=None) -> np.ndarray:
    """Return the grid after T steps (u is not modified). lib: an alternative library from load().

    field: optional per-point weights of shape (K,) + grid shape in canonical term order; it
    replaces the constant weights (which still give K).
    """
    lib = lib if lib is not None else _load()
    a = np.array(u, dtype=np.float64, order="C", copy=True)
    if a.ndim != dim:
        raise ValueError("grid rank %d != dim %d" % (a.ndim, dim))
    w = np.ascontiguousarray(weights, dtype=np.float64)
    ext = (ctypes.c_int64 * 3)(*(list(a.shape) + [1] * (3 - dim)))
    dptr = ctypes.POINTER(ctypes.c_double)
    if field is None:
        rc = lib.oracle_run(dim, shape, r, w.ctypes.data_as(dptr), len(w), method, bc, float(c), arith, ext, int(T),
                            a.ctypes.data_as(dptr), int(nthreads))
    else:
        f = np.ascontiguousarray(field, dtype=np.float64)
        if f.shape != (len(w),) + a.shape:
            raise ValueError("field must have shape (K,) + grid shape")
        rc = lib.oracle_run_field(dim, shape, r, w.ctypes.data_as(dptr), f.ctypes.data_as(dptr), len(w), method, bc,
                                  float(c), arith, ext, int(T), a.ctypes.data_as(dptr), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_run rejected its arguments")
    return a
