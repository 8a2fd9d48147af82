"""CPU oracle for the integer stencils (Game of Life and LCS, Section 3.4).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark legs that time the oracle use it; the library never does. It shares
no code with the CUDA path and never imports it.

``life`` calls the plain C definition in ``int_oracle.c``: two arrays, every
cell's 8 neighbours counted from the previous step, the birth/survival rule
applied by table lookup in the rule's bit masks. ``lcs`` calls the textbook
dynamic program for the longest common subsequence, one row updated in
place over B for every character of A.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

BC_CONSTANT, BC_PERIODIC = 0, 1
#: The paper's variant B2S23: born with 2 live neighbours, survives with 2 or 3.
B2S23 = (1 << 2, (1 << 2) | (1 << 3))
#: Conway's rule B3S23 (for textbook patterns).
B3S23 = (1 << 3, (1 << 2) | (1 << 3))

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "int_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_int.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the integer oracle with gcc (-O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def load(path: str):
    lib = ctypes.CDLL(path)
    lib.oracle_life.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                ctypes.c_int64, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int]
    lib.oracle_life.restype = ctypes.c_int
    if hasattr(lib, "oracle_lcs"):
        lib.oracle_lcs.argtypes = [ctypes.POINTER(ctypes.c_uint8), ctypes.c_int64, ctypes.POINTER(ctypes.c_uint8),
                                   ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]
        lib.oracle_lcs.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def life(cells, T: int, *, bc: int = BC_CONSTANT, rule=B2S23, nthreads: int = 0, lib=None) -> np.ndarray:
    """Return the 2D 0/1 grid after T steps (cells is not modified). rule = (birth_mask, survive_mask)."""
    lib = lib if lib is not None else _load()
    a = np.array(cells, dtype=np.uint8, order="C", copy=True)
    if a.ndim != 2:
        raise ValueError("life grids are 2D")
    rc = lib.oracle_life(a.shape[0], a.shape[1], int(bc), int(rule[0]), int(rule[1]), int(T),
                         a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_life rejected its arguments")
    return a


def lcs(A, B, lib=None) -> np.ndarray:
    """Row lcs[len(A)][0..len(B)] of the LCS dynamic program (int32); its last entry is the LCS length."""
    lib = lib if lib is not None else _load()
    a = np.ascontiguousarray(np.frombuffer(bytes(A), np.uint8) if isinstance(A, (bytes, bytearray)) else A,
                             dtype=np.uint8)
    b = np.ascontiguousarray(np.frombuffer(bytes(B), np.uint8) if isinstance(B, (bytes, bytearray)) else B,
                             dtype=np.uint8)
    row = np.zeros(len(b) + 1, np.int32)
    P8 = ctypes.POINTER(ctypes.c_uint8)
    rc = lib.oracle_lcs(a.ctypes.data_as(P8), len(a), b.ctypes.data_as(P8), len(b),
                        row.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc != 0:
        raise ValueError("oracle_lcs rejected its arguments")
    return row
