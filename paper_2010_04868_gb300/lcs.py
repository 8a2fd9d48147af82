"""Python binding of the LCS entry points (include/lcs.h): argument marshalling only.

Longest common subsequence (Section 3.4) as a 1D Gauss-Seidel wavefront over the rows of A; the
kernels run in the CUDA library, this module passes pointers and lengths through the C ABI.
"""
from __future__ import annotations

import ctypes

from . import stencil as S

LCS_KERNEL_AUTO, LCS_KERNEL_DP, LCS_KERNEL_BITS = 0, 1, 2


def lcs_workspace_bytes(na, nb, kernel=LCS_KERNEL_AUTO) -> int:
    b = ctypes.c_size_t()
    S.check(S.load().lcs_workspace_bytes(int(na), int(nb), int(kernel), ctypes.byref(b)), "lcs_workspace_bytes")
    return b.value


def lcs_run(a_ptr, na, b_ptr, nb, row_ptr, kernel=LCS_KERNEL_AUTO, workspace_ptr=None, stream_ptr=None):
    return S.check(S.load().lcs_run(a_ptr, int(na), b_ptr, int(nb), row_ptr, int(kernel), workspace_ptr, stream_ptr),
                   "lcs_run")


def lcs_status(workspace_ptr, stream_ptr=None) -> int:
    return S.load().lcs_status(workspace_ptr, stream_ptr)


def run(A, B, kernel=LCS_KERNEL_AUTO, row=None, workspace=None, stream=None):
    """A, B: contiguous 1D uint8 CUDA tensors. Returns the int32 CUDA tensor row[y] = lcs[len(A)][y], y = 0..len(B)."""
    import torch
    for name, t in (("A", A), ("B", B)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.uint8 and t.is_contiguous()
                and t.dim() == 1):
            raise ValueError("%s must be a contiguous 1D uint8 CUDA tensor" % name)
    if row is None:
        row = torch.empty(B.numel() + 1, dtype=torch.int32, device=B.device)
    ws = None
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < lcs_workspace_bytes(A.numel(), B.numel(), kernel):
            raise ValueError("workspace too small")
        ws = workspace.data_ptr()
    lcs_run(A.data_ptr() if A.numel() else None, A.numel(), B.data_ptr() if B.numel() else None, B.numel(),
            row.data_ptr(), kernel, ws, S._stream_ptr(stream))
    return row
