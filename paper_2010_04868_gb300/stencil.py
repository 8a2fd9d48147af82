"""Python binding of the stencil library's C ABI (include/stencil.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. The function names follow the C ABI; ``Stencil`` is a small
convenience wrapper taking torch tensors (float64, CUDA, contiguous) and
torch streams. PyTorch provides device memory and streams, nothing else.
Loading fails loudly (``RuntimeError``) when the built library is missing.
"""
from __future__ import annotations

import ctypes
import os

STENCIL_OK = 0
STENCIL_EINVAL = -1
STENCIL_EUNSUPPORTED = -2
STENCIL_ENOMEM = -3
STENCIL_ECUDA = -4
STENCIL_ETIMEOUT = -5
STENCIL_EBOUNDS = -6

STENCIL_STAR, STENCIL_BOX = 0, 1
STENCIL_JACOBI, STENCIL_GAUSS_SEIDEL = 0, 1
STENCIL_BC_CONSTANT, STENCIL_BC_PERIODIC = 0, 1
STENCIL_ARITH_FMA, STENCIL_ARITH_UNFUSED = 0, 1
STENCIL_KERNEL_AUTO, STENCIL_KERNEL_PLAIN, STENCIL_KERNEL_BLOCKED, STENCIL_KERNEL_WAVEFRONT = 0, 1, 2, 3
STENCIL_KERNEL_DIAMOND = 4
STENCIL_KERNEL_STREAM = 5

#: The library this module loads: the checked build (every kernel index tested before its access, a
#: failing test reported as STENCIL_EBOUNDS) when the environment sets STENCIL_CHECKED=1, else the normal one.
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "libgb300stencil_checked.so" if os.environ.get("STENCIL_CHECKED") == "1"
                        else "libgb300stencil.so")

#: Every entry point that include/stencil.h declares.
EXPORTS = ("stencil_create", "stencil_set_plan", "stencil_run", "stencil_run_batch", "stencil_workspace_bytes",
           "stencil_status", "stencil_destroy", "stencil_strerror", "stencil_run_host", "stencil_launch_count",
           "stencil_run_noalloc", "stencil_debug_inject_stall", "stencil_set_coeff_field", "stencil_get_plan",
           "life_workspace_bytes", "life_run", "lcs_workspace_bytes", "lcs_run", "lcs_status",
           "stencil_checked_build", "stencil_debug_check_index")

#: Largest grid (points) stencil_run_noalloc accepts: its fixed workspace holds 2^21 doubles.
NOALLOC_MAX_POINTS = 1 << 21


class stencil_grid(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("ext", ctypes.c_int64 * 3), ("scratch", ctypes.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library and declare its signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("CUDA stencil library not built: %s (run __graft_entry__.build())" % path)
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.stencil_create.argtypes = [I, I, I, ctypes.POINTER(D), I, I, I, D, I, ctypes.POINTER(P)]
    lib.stencil_set_plan.argtypes = [P, I, I, ctypes.POINTER(I64)]
    lib.stencil_run.argtypes = [P, ctypes.POINTER(stencil_grid), I64, P]
    lib.stencil_run_batch.argtypes = [ctypes.POINTER(P), ctypes.POINTER(stencil_grid), ctypes.POINTER(I64), I, P]
    lib.stencil_workspace_bytes.argtypes = [P, ctypes.POINTER(stencil_grid), ctypes.POINTER(ctypes.c_size_t)]
    lib.stencil_status.argtypes = [P, P]
    lib.stencil_destroy.argtypes = [P]
    lib.stencil_strerror.argtypes = [I]
    lib.stencil_strerror.restype = ctypes.c_char_p
    lib.stencil_run_host.argtypes = [P, P, ctypes.POINTER(I64), P, P, I64, P]
    lib.stencil_run_noalloc.argtypes = [P, ctypes.POINTER(stencil_grid), I64, P]
    lib.stencil_debug_inject_stall.argtypes = [P, I64, I]
    lib.stencil_set_coeff_field.argtypes = [P, P, ctypes.POINTER(I64)]
    lib.stencil_get_plan.argtypes = [P, ctypes.POINTER(stencil_grid), I64, P, ctypes.POINTER(I), ctypes.POINTER(I),
                                     ctypes.POINTER(I64)]
    lib.life_workspace_bytes.argtypes = [ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_size_t)]
    lib.life_run.argtypes = [P, ctypes.POINTER(I64), I, ctypes.c_uint32, ctypes.c_uint32, I64, I, P, P]
    lib.lcs_workspace_bytes.argtypes = [I64, I64, I, ctypes.POINTER(ctypes.c_size_t)]
    lib.lcs_run.argtypes = [P, I64, P, I64, P, I, P, P]
    lib.lcs_status.argtypes = [P, P]
    lib.stencil_launch_count.argtypes = []
    lib.stencil_checked_build.argtypes = []
    lib.stencil_debug_check_index.argtypes = [I64, I64, P]
    lib.stencil_launch_count.restype = ctypes.c_uint64
    for name in EXPORTS:
        if name not in ("stencil_strerror", "stencil_launch_count"):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().stencil_strerror(int(code)).decode()


class StencilError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (%d)" % (what, strerror(code), code))
        self.code = code


def check(code: int, what: str = "stencil call") -> int:
    if code != STENCIL_OK:
        raise StencilError(code, what)
    return code


# ---- thin wrappers with the C names -------------------------------------------------------

def stencil_create(dim, shape, radius, coeffs, method, boundary, boundary_value=0.0, arith=STENCIL_ARITH_FMA):
    lib = load()
    arr = (ctypes.c_double * len(coeffs))(*[float(x) for x in coeffs])
    h = ctypes.c_void_p()
    check(lib.stencil_create(int(dim), int(shape), int(radius), arr, len(coeffs), int(method), int(boundary),
                             float(boundary_value), int(arith), ctypes.byref(h)), "stencil_create")
    return h


def stencil_set_plan(h, kernel, tb=0, tile=(0, 0, 0)):
    t = (ctypes.c_int64 * 3)(*[int(x) for x in tile])
    return check(load().stencil_set_plan(h, int(kernel), int(tb), t), "stencil_set_plan")


def make_grid(data_ptr, ext, scratch_ptr=None):
    e = list(ext) + [1] * (3 - len(ext))
    return stencil_grid(data_ptr, (ctypes.c_int64 * 3)(*e), scratch_ptr)


def stencil_run(h, grid: stencil_grid, T, stream_ptr=None):
    return check(load().stencil_run(h, ctypes.byref(grid), int(T), stream_ptr), "stencil_run")


def stencil_run_batch(handles, grids, Ts, stream_ptr=None):
    n = len(handles)
    H = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    G = (stencil_grid * n)(*grids)
    T = (ctypes.c_int64 * n)(*[int(t) for t in Ts])
    return check(load().stencil_run_batch(H, G, T, n, stream_ptr), "stencil_run_batch")


def stencil_set_coeff_field(h, field_ptr, ext):
    """Bind per-point weights (device pointer to K x N doubles, canonical term-major); None unbinds."""
    e = (ctypes.c_int64 * 3)(*(list(ext) + [1] * (3 - len(ext))))
    return check(load().stencil_set_coeff_field(h, field_ptr, e), "stencil_set_coeff_field")


def stencil_get_plan(h, grid: stencil_grid, T, stream_ptr=None):
    """(kernel, tb, tile) that stencil_run would use for this grid and T (tuning first if needed)."""
    k, tb = ctypes.c_int(), ctypes.c_int()
    tile = (ctypes.c_int64 * 3)()
    check(load().stencil_get_plan(h, ctypes.byref(grid), int(T), stream_ptr, ctypes.byref(k), ctypes.byref(tb), tile),
          "stencil_get_plan")
    return k.value, tb.value, tuple(tile)


def stencil_workspace_bytes(h, grid: stencil_grid) -> int:
    b = ctypes.c_size_t()
    check(load().stencil_workspace_bytes(h, ctypes.byref(grid), ctypes.byref(b)), "stencil_workspace_bytes")
    return b.value


def stencil_status(h, stream_ptr=None) -> int:
    return load().stencil_status(h, stream_ptr)


def stencil_destroy(h):
    return check(load().stencil_destroy(h), "stencil_destroy")


def stencil_run_host(h, host_ptr, ext, dev_data_ptr, dev_scratch_ptr, T, stream_ptr=None):
    e = (ctypes.c_int64 * 3)(*(list(ext) + [1] * (3 - len(ext))))
    return check(load().stencil_run_host(h, host_ptr, e, dev_data_ptr, dev_scratch_ptr, int(T), stream_ptr),
                 "stencil_run_host")


def stencil_run_noalloc(h, grid: stencil_grid, T, stream_ptr=None):
    """Jacobi run whose workspace is the library's fixed 16 MiB array: no device allocation.

    For callers that may not allocate device memory. Grids above
    NOALLOC_MAX_POINTS points are rejected; calls that overlap on the GPU race
    on the shared array.
    """
    rc = load().stencil_run_noalloc(h, ctypes.byref(grid), int(T), stream_ptr)
    if rc == STENCIL_EUNSUPPORTED:
        npts = 1
        for e in grid.ext:
            npts *= max(1, int(e))
        raise StencilError(rc, "stencil_run_noalloc: grid of %d points exceeds the %d-point no-allocation "
                               "workspace (or the handle is not supported)" % (npts, NOALLOC_MAX_POINTS))
    return check(rc, "stencil_run_noalloc")


def stencil_debug_inject_stall(h, unit, spin=0):
    """Failure-detection test hook: the next wavefront run never publishes work unit `unit`."""
    return check(load().stencil_debug_inject_stall(h, int(unit), int(spin)), "stencil_debug_inject_stall")


def stencil_launch_count() -> int:
    return int(load().stencil_launch_count())


def checked_build() -> bool:
    """True if the loaded library is the checked build."""
    return bool(load().stencil_checked_build())


def debug_check_index(i: int, n: int, stream=None) -> int:
    """Run the checked build's index test of i against n in one device thread (no memory access)."""
    return load().stencil_debug_check_index(int(i), int(n), _stream_ptr(stream))


# ---- torch convenience ---------------------------------------------------------------------

def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_tensor(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)


class Stencil:
    """A stencil handle. run() advances a CUDA float64 tensor in place on a torch stream."""

    def __init__(self, dim, shape, radius, coeffs, method=STENCIL_JACOBI, boundary=STENCIL_BC_CONSTANT,
                 boundary_value=0.0, arith=STENCIL_ARITH_FMA):
        self.dim, self.method = int(dim), int(method)
        self.handle = stencil_create(dim, shape, radius, coeffs, method, boundary, boundary_value, arith)

    def set_plan(self, kernel, tb=0, tile=(0, 0, 0)):
        stencil_set_plan(self.handle, kernel, tb, tile)
        return self

    def set_field(self, field):
        """Bind per-point weights: a float64 CUDA tensor of shape (K,) + grid shape, canonical term order
        (None unbinds). The handle keeps a reference so the memory outlives the binding."""
        if field is None:
            stencil_set_coeff_field(self.handle, None, (0, 0, 0))
            self._field = None
            return self
        _check_tensor(field, "field")
        if field.dim() != self.dim + 1:
            raise ValueError("field must have shape (K,) + grid shape")
        stencil_set_coeff_field(self.handle, field.data_ptr(), tuple(field.shape[1:]))
        self._field = field
        return self

    def grid(self, u, scratch=None):
        _check_tensor(u, "u")
        if u.dim() != self.dim:
            raise ValueError("tensor rank %d != stencil dim %d" % (u.dim(), self.dim))
        if scratch is not None:
            _check_tensor(scratch, "scratch")
            if scratch.numel() < u.numel():
                raise ValueError("scratch too small")
        return make_grid(u.data_ptr(), tuple(u.shape), scratch.data_ptr() if scratch is not None else None)

    def run(self, u, T, scratch=None, stream=None):
        stencil_run(self.handle, self.grid(u, scratch), T, _stream_ptr(stream))
        return u

    def plan(self, u, T, stream=None):
        """(kernel, tb, tile) that run(u, T) would use."""
        return stencil_get_plan(self.handle, self.grid(u), T, _stream_ptr(stream))

    def status(self, stream=None) -> int:
        return stencil_status(self.handle, _stream_ptr(stream))

    def close(self):
        if self.handle is not None:
            stencil_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
