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
from paper_2010_04868_gb300 import inputs

pytestmark = pytest.mark.gpu


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _run_reference(S, h, u0, T):
    import torch
    u = torch.from_numpy(u0.copy()).cuda()
    scratch = torch.empty_like(u)
    S.stencil_run(h, S.make_grid(u.data_ptr(), u0.shape, scratch.data_ptr()), T, _stream())
    torch.cuda.synchronize()
    return u.cpu().numpy()


def _run_noalloc(S, h, u0, T):
    import torch
    u = torch.from_numpy(u0.copy()).cuda()
    S.stencil_run_noalloc(h, S.make_grid(u.data_ptr(), u0.shape, None), T, _stream())
    torch.cuda.synchronize()
    return u.cpu().numpy()


def _compare_two_calls(S, h, u0, T):
    S.stencil_set_plan(h, S.STENCIL_KERNEL_PLAIN)
    ref = _run_reference(S, h, u0, T)
    for _ in range(2):                      # the second call finds the first call's leftovers in the array
        got = _run_noalloc(S, h, u0, T)
        assert bits_equal(got, ref), first_diff(got, ref)
    assert S.stencil_status(h, _stream()) == 0


@pytest.mark.parametrize("dim,shape,ext,T,bc", [(2, "star", (300, 257), 7, 0), (3, "box", (40, 33, 64), 4, 0),
                                                (1, "star", (100003,), 9, 0), (2, "box", (129, 77), 6, 1),
                                                (3, "star", (24, 17, 40), 5, 1)])
def test_noalloc_matches_stencil_run_on_two_calls(dim, shape, ext, T, bc):
    from paper_2010_04868_gb300 import stencil as S
    w, u0 = case(dim, shape, 1, ext, seed=dim + 40 + 7 * bc)
    h = S.stencil_create(dim, 0 if shape == "star" else 1, 1, list(w), S.STENCIL_JACOBI, bc, 0.25)
    _compare_two_calls(S, h, u0, T)
    S.stencil_destroy(h)


def test_noalloc_with_coefficient_field_matches_stencil_run():
    import torch
    from paper_2010_04868_gb300 import stencil as S
    ext = (61, 90)
    f = torch.from_numpy(inputs.normalized_field(4401, 9, ext)).cuda()
    u0 = inputs.grid(4402, ext)
    h = S.stencil_create(2, 1, 1, [0.0] * 9, S.STENCIL_JACOBI, S.STENCIL_BC_CONSTANT, 0.5)
    S.stencil_set_coeff_field(h, f.data_ptr(), ext)
    _compare_two_calls(S, h, u0, 5)
    S.stencil_destroy(h)


def test_noalloc_rejects_without_launching():
    """Every rejected call passes T = 0: were a check to let it through, nothing would run."""
    from paper_2010_04868_gb300 import stencil as S
    h = S.stencil_create(1, 0, 1, [0.25, 0.5, 0.25], S.STENCIL_JACOBI, S.STENCIL_BC_CONSTANT, 0.0)
    h2 = S.stencil_create(2, 0, 1, [0.2] * 5, S.STENCIL_JACOBI, S.STENCIL_BC_CONSTANT, 0.0)
    h3 = S.stencil_create(3, 0, 1, [1 / 7] * 7, S.STENCIL_JACOBI, S.STENCIL_BC_CONSTANT, 0.0)
    gs = S.stencil_create(1, 0, 1, [0.25, 0.5, 0.25], S.STENCIL_GAUSS_SEIDEL, S.STENCIL_BC_CONSTANT, 0.0)
    fake = 1 << 20                                          # never dereferenced: every case is rejected first
    cases = [(h, (S.NOALLOC_MAX_POINTS + 1,), S.STENCIL_EUNSUPPORTED),
             (h2, (2048, 1025), S.STENCIL_EUNSUPPORTED),
             (h3, (128, 128, 129), S.STENCIL_EUNSUPPORTED),
             (h2, (4, 1 << 62), S.STENCIL_EINVAL),           # the product of the extents overflows
             (h2, (2, 1 << 62), S.STENCIL_EINVAL),
             (h3, (2, 2, 1 << 62), S.STENCIL_EINVAL),
             (h3, (1 << 40, 1 << 40, 1 << 40), S.STENCIL_EINVAL),
             (h2, (0, 5), S.STENCIL_EINVAL),
             (gs, (100,), S.STENCIL_EINVAL)]                 # Gauss-Seidel works in place: not this entry point
    for hh, ext, code in cases:
        with pytest.raises(S.StencilError) as e:
            S.stencil_run_noalloc(hh, S.make_grid(fake, ext, None), 0, _stream())
        assert e.value.code == code, (ext, e.value.code)
    for hh in (h, h2, h3, gs):
        S.stencil_destroy(hh)
