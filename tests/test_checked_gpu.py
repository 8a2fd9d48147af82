"""The checked build (libgb300stencil_checked.so: every kernel index tested before its access, a
failing test reported as STENCIL_EBOUNDS instead of touching memory) on the parity suites' small,
ragged cases of every kernel family: each run reports STENCIL_OK and equals the oracle bit for bit.

The index-check hook (stencil_debug_check_index) shows that a failing test is reported, and
cleared by the status read, without any out-of-range access being made.
"""
import ctypes

import numpy as np
import pytest

from helpers import bits_equal, case, first_diff, gpu_run, oracle_run
import test_batch_gpu as tb_
import test_parity_blocked_gpu as tbl
import test_parity_diamond_gpu as tdi
import test_parity_plain_gpu as tpl
import test_parity_stream_gpu as tst
import test_parity_wavefront_gpu as twf

pytestmark = pytest.mark.gpu

PLAIN, BLOCKED, WAVE, DIAMOND, STREAM = 1, 2, 3, 4, 5


@pytest.fixture(scope="module", autouse=True)
def checked_library():
    """Route every call of this module through the checked build, then restore the normal library."""
    from paper_2010_04868_gb300 import build, stencil as S
    build.build()
    saved = S._lib
    S._lib = None
    S.load(build.LIB_CHECKED)
    assert S.checked_build()
    yield
    S._lib = saved


def _stream():
    import torch
    return torch.cuda.current_stream()


def test_index_hook_reports_and_clears():
    from paper_2010_04868_gb300 import stencil as S
    st = S.Stencil(1, 0, 1, [0.25, 0.5, 0.25], S.STENCIL_JACOBI)
    for i, n, want in ((5, 10, S.STENCIL_OK), (10, 10, S.STENCIL_EBOUNDS), (0, 1, S.STENCIL_OK),
                       (-1, 10, S.STENCIL_EBOUNDS), (1 << 40, 1 << 41, S.STENCIL_OK)):
        assert S.debug_check_index(i, n, _stream()) == S.STENCIL_OK
        assert st.status() == want, (i, n)
    assert st.status() == S.STENCIL_OK          # the record was cleared by the read that reported it
    st.close()


def _check(u0, T, dim, shape, r, w, method, bc, c, plan, tb=0, tile=(0, 0, 0), scratch=True):
    ref = oracle_run(u0, T, dim, shape, r, w, method, bc, c, "fma")
    got = gpu_run(u0, T, dim, shape, r, w, method, bc, c, "fma", plan=plan, tb=tb, tile=tile, use_scratch=scratch)
    assert bits_equal(got, ref), first_diff(got, ref)


BCS = [("constant", 0.3), ("periodic", 0.0)]


def _periodic_ok(bc, ext, r):
    return bc != "periodic" or min(ext) >= 2 * r + 1


@pytest.mark.parametrize("dim,shape,r,ext", tpl.JACOBI_CASES)
@pytest.mark.parametrize("bc,c", BCS)
def test_checked_jacobi_plain(dim, shape, r, ext, bc, c):
    if not _periodic_ok(bc, ext, r):
        pytest.skip("periodic needs ext >= 2r+1")
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r)
    _check(u0, 3, dim, shape, r, w, "jacobi", bc, c, PLAIN)


@pytest.mark.parametrize("dim,shape,r,ext", tpl.GS_CASES)
@pytest.mark.parametrize("bc,c", BCS)
def test_checked_gs_plain(dim, shape, r, ext, bc, c):
    if not _periodic_ok(bc, ext, r):
        pytest.skip("periodic needs ext >= 2r+1")
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r + 1)
    _check(u0, 2, dim, shape, r, w, "gs", bc, c, PLAIN)


@pytest.mark.parametrize("dim,shape,r,ext,tb,tile", tst.CASES)
@pytest.mark.parametrize("bc,c", BCS)
def test_checked_stream(dim, shape, r, ext, tb, tile, bc, c):
    if not _periodic_ok(bc, ext, r):
        pytest.skip("periodic needs ext >= 2r+1")
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r + 5)
    _check(u0, 3 * tb + 2, dim, shape, r, w, "jacobi", bc, c, STREAM, tb=tb, tile=tile)


@pytest.mark.parametrize("dim,shape,r,ext,tb,tile", tbl.CASES)
@pytest.mark.parametrize("bc,c", BCS)
def test_checked_blocked(dim, shape, r, ext, tb, tile, bc, c):
    if not _periodic_ok(bc, ext, r):
        pytest.skip("periodic needs ext >= 2r+1")
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r + 5)
    _check(u0, 2 * tb + 1, dim, shape, r, w, "jacobi", bc, c, BLOCKED, tb=tb, tile=tile)


@pytest.mark.parametrize("dim,shape,r,ext,H,periods", tdi.CASES)
@pytest.mark.parametrize("bc,c", BCS)
def test_checked_diamond(dim, shape, r, ext, H, periods, bc, c):
    if not _periodic_ok(bc, ext, r) or min(ext) < 2 * r:
        pytest.skip("periodic needs ext >= 2r+1; split tiles need ext >= 2r")
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r + 5)
    _check(u0, 2 * H + 1, dim, shape, r, w, "jacobi", bc, c, DIAMOND, tb=H, tile=periods, scratch=False)


@pytest.mark.parametrize("dim,shape,r,ext", twf.CASES_ND)
def test_checked_wavefront_nd(dim, shape, r, ext):
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r + 3)
    _check(u0, 37, dim, shape, r, w, "gs", "constant", 0.3, WAVE)


@pytest.mark.parametrize("dim,r,ext", twf.PERIODIC_CASES)
def test_checked_wavefront_periodic(dim, r, ext):
    w, u0 = case(dim, "star", r, ext, seed=dim * 10 + r + 4)
    _check(u0, 5, dim, "star", r, w, "gs", "periodic", 0.0, WAVE)


@pytest.mark.parametrize("r,n", [(1, 3000), (1, 37), (2, 1000)])
def test_checked_wavefront_1d(r, n):
    w, u0 = case(1, "star", r, (n,), seed=r + 40)
    _check(u0, 45, 1, "star", r, w, "gs", "constant", 0.2, WAVE)


def test_checked_batch_mix():
    import torch
    from paper_2010_04868_gb300 import stencil as S
    sts, grids, Ts, tensors, refs = tb_._setup(tb_.MIX)
    S.stencil_run_batch([s.handle for s in sts], grids, Ts, ctypes.c_void_p(_stream().cuda_stream))
    torch.cuda.synchronize()
    for n, (st, (u, _, _), ref) in enumerate(zip(sts, tensors, refs)):
        assert st.status() == S.STENCIL_OK, n
        got = u.cpu().numpy()
        assert bits_equal(got, ref), (n, tb_.MIX[n], first_diff(got, ref))
    for st in sts:
        st.close()


@pytest.mark.parametrize("dim,method,plan,ext", [(2, "jacobi", PLAIN, (67, 45)), (3, "jacobi", PLAIN, (9, 10, 21)),
                                                 (2, "gs", WAVE, (50, 61)), (1, "gs", WAVE, (2000,)),
                                                 (2, "gs", PLAIN, (40, 33))])
def test_checked_coefficient_field(dim, method, plan, ext):
    import torch
    import oracle
    from paper_2010_04868_gb300 import inputs, stencil as S
    k = 2 * dim + 1
    field = inputs.normalized_field(77 + dim, k, ext)
    u0 = inputs.grid(78 + dim, ext)
    m = 0 if method == "jacobi" else 1
    ref = oracle.run(u0, 4, dim=dim, shape=0, r=1, weights=[0.0] * k, method=m, bc=0, c=0.1, arith=0, field=field)
    st = S.Stencil(dim, 0, 1, [1.0] * k, m, 0, 0.1, 0).set_plan(plan)
    st.set_field(torch.from_numpy(np.ascontiguousarray(field)).cuda())
    u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    st.run(u, 4, torch.empty_like(u) if m == 0 else None)
    assert st.status() == S.STENCIL_OK
    got = u.cpu().numpy()
    st.close()
    assert bits_equal(got, ref), first_diff(got, ref)


@pytest.mark.parametrize("shape,r,ext", [("star", 1, (70, 44)), ("box", 1, (33, 68)), ("star", 2, (97, 36)),
                                         ("star", 1, (1, 8))])
def test_checked_wavefront_rows(shape, r, ext):
    """The 2D wavefront's default plan on whole groups of four columns: rows as lanes."""
    w, u0 = case(2, shape, r, ext, seed=ext[0] + r)
    _check(u0, 9, 2, shape, r, w, "gs", "constant", 0.3, WAVE)


def test_checked_wavefront_rows_field():
    import torch
    import oracle
    from paper_2010_04868_gb300 import inputs, stencil as S
    ext = (45, 64)
    field = inputs.normalized_field(91, 5, ext)
    u0 = inputs.grid(92, ext)
    ref = oracle.run(u0, 6, dim=2, shape=0, r=1, weights=[0.0] * 5, method=1, bc=0, c=0.1, arith=0, field=field)
    st = S.Stencil(2, 0, 1, [1.0] * 5, 1, 0, 0.1, 0).set_plan(WAVE)
    st.set_field(torch.from_numpy(np.ascontiguousarray(field)).cuda())
    u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    st.run(u, 6)
    assert st.status() == S.STENCIL_OK
    got = u.cpu().numpy()
    st.close()
    assert bits_equal(got, ref), first_diff(got, ref)
