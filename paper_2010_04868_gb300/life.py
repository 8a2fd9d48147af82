"""Python binding of the Game of Life entry points (include/life.h): argument marshalling only.

Game of Life (Section 3.4): a 2D Jacobi stencil over the 3 x 3 box on 0/1 cells. The library
packs the cells into bits and runs every step in its CUDA kernels; this module passes pointers,
extents and the rule through the C ABI.
"""
from __future__ import annotations

import ctypes

from . import stencil as S

#: The paper's variant B2S23: born with 2 live neighbours, survives with 2 or 3.
B2S23 = (1 << 2, (1 << 2) | (1 << 3))
#: Conway's rule B3S23.
B3S23 = (1 << 3, (1 << 2) | (1 << 3))


def _ext(ext):
    return (ctypes.c_int64 * 2)(int(ext[0]), int(ext[1]))


def life_workspace_bytes(ext) -> int:
    b = ctypes.c_size_t()
    S.check(S.load().life_workspace_bytes(_ext(ext), ctypes.byref(b)), "life_workspace_bytes")
    return b.value


def life_run(cells_ptr, ext, T, boundary=S.STENCIL_BC_CONSTANT, rule=B2S23, tb=0, workspace_ptr=None,
             stream_ptr=None):
    return S.check(S.load().life_run(cells_ptr, _ext(ext), int(boundary), int(rule[0]), int(rule[1]), int(T),
                                     int(tb), workspace_ptr, stream_ptr), "life_run")


def run(cells, T, boundary=S.STENCIL_BC_CONSTANT, rule=B2S23, tb=0, workspace=None, stream=None):
    """Advance a contiguous uint8 CUDA tensor of shape (n0, n1) in place by T steps on a torch stream."""
    import torch
    if not (isinstance(cells, torch.Tensor) and cells.is_cuda and cells.dtype == torch.uint8
            and cells.is_contiguous() and cells.dim() == 2):
        raise ValueError("cells must be a contiguous 2D uint8 CUDA tensor")
    ws = None
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < life_workspace_bytes(cells.shape):
            raise ValueError("workspace too small")
        ws = workspace.data_ptr()
    life_run(cells.data_ptr(), tuple(cells.shape), T, boundary, rule, tb, ws, S._stream_ptr(stream))
    return cells
