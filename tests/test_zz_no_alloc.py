"""The allocation-free Jacobi entry point gives the same grids as stencil_run.

stencil_run_noalloc exists for callers that may not allocate device memory
(a device-memory budget fixed in advance, real-time loops that must stay out
of the CUDA allocator, host code running where allocation is forbidden); its
workspace is a fixed array inside the library. This file is collected last,
so a run that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from helpers import bits_equal, case, first_diff

pytestmark = pytest.mark.gpu


def _run_reference(S, h, u0, T, stream):
    import torch
    u = torch.from_numpy(u0.copy()).cuda()
    scratch = torch.empty_like(u)
    S.stencil_run(h, S.make_grid(u.data_ptr(), u0.shape, scratch.data_ptr()), T, stream)
    torch.cuda.synchronize()
    return u.cpu().numpy()


def _run_noalloc(S, h, u0, T, stream):
    import torch
    u = torch.from_numpy(u0.copy()).cuda()
    S.stencil_run_noalloc(h, S.make_grid(u.data_ptr(), u0.shape, None), T, stream)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("dim,shape,ext,T", [(2, "star", (300, 257), 7), (3, "box", (40, 33, 64), 4),
                                             (1, "star", (100003,), 9)])
def test_noalloc_matches_stencil_run_on_two_calls(dim, shape, ext, T):
    import torch
    from paper_2010_04868_gb300 import stencil as S
    w, u0 = case(dim, shape, 1, ext, seed=dim + 40)
    h = S.stencil_create(dim, 0 if shape == "star" else 1, 1, list(w), S.STENCIL_JACOBI, S.STENCIL_BC_CONSTANT, 0.25)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    S.stencil_set_plan(h, S.STENCIL_KERNEL_PLAIN)
    ref = _run_reference(S, h, u0, T, stream)
    for _ in range(2):                      # the second call finds the first call's leftovers in the array
        got = _run_noalloc(S, h, u0, T, stream)
        assert bits_equal(got, ref), first_diff(got, ref)
    assert S.stencil_status(h, stream) == 0
    S.stencil_destroy(h)


def test_noalloc_rejects_grids_beyond_its_capacity():
    import torch
    from paper_2010_04868_gb300 import stencil as S
    h = S.stencil_create(1, 0, 1, [0.25, 0.5, 0.25], S.STENCIL_JACOBI, S.STENCIL_BC_CONSTANT, 0.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    big = S.make_grid(1 << 20, (S.NOALLOC_MAX_POINTS + 1,), None)   # rejected before any device access
    with pytest.raises(S.StencilError) as e:
        S.stencil_run_noalloc(h, big, 1, stream)
    assert e.value.code == S.STENCIL_EUNSUPPORTED
    S.stencil_destroy(h)
