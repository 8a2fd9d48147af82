"""Variable-coefficient stencils (per-point weights, Section 3.4's variable coefficient): the CUDA
kernels against the oracle, bit for bit, through the C ABI."""
import ctypes

import numpy as np
import pytest

from helpers import ARITH_ID, BC_ID, METHOD_ID, SHAPE_ID, bits_equal, first_diff, k_of
import oracle
from paper_2010_04868_gb300 import inputs

pytestmark = pytest.mark.gpu

PLAIN, BLOCKED, WAVE = 1, 2, 3


def _case(dim, shape, r, ext, seed):
    k = k_of(dim, shape, r)
    return inputs.normalized_field(seed, k, ext), inputs.grid(seed + 1, ext), k


def _oracle(u0, T, dim, shape, r, field, method, bc, c, arith):
    k = field.shape[0]
    return oracle.run(u0, T, dim=dim, shape=SHAPE_ID[shape] if dim > 1 else 0, r=r, weights=[0.0] * k,
                      method=METHOD_ID[method], bc=BC_ID[bc], c=c, arith=ARITH_ID[arith], field=field)


def _gpu(u0, T, dim, shape, r, field, method, bc, c, arith, plan=None):
    import torch
    from paper_2010_04868_gb300 import stencil as S
    k = field.shape[0]
    # the constant weights are deliberately wrong: a kernel that ignores the field fails
    st = S.Stencil(dim, SHAPE_ID[shape], r, [1.0] * k, METHOD_ID[method], BC_ID[bc], c, ARITH_ID[arith])
    if plan is not None:
        st.set_plan(plan)
    st.set_field(torch.from_numpy(np.ascontiguousarray(field)).cuda())
    u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    scratch = torch.empty_like(u) if method == "jacobi" else None
    st.run(u, T, scratch)
    rc = st.status()
    assert rc == 0, S.strerror(rc)
    out = u.cpu().numpy()
    st.close()
    return out


JACOBI_CASES = [
    (1, "star", 1, (1,)), (1, "star", 1, (1000,)), (1, "star", 2, (333,)), (1, "star", 3, (97,)),
    (2, "star", 1, (37, 130)), (2, "box", 1, (70, 131)), (2, "star", 2, (64, 65)), (2, "box", 2, (33, 70)),
    (3, "star", 1, (9, 10, 21)), (3, "box", 1, (9, 10, 21)), (3, "star", 2, (12, 11, 13)),
    (3, "box", 2, (7, 8, 9)),     # no compile-time specialisation: the run-time offset kernel
]


@pytest.mark.parametrize("dim,shape,r,ext", JACOBI_CASES)
@pytest.mark.parametrize("bc", ["constant", "periodic"])
def test_jacobi_field(dim, shape, r, ext, bc):
    if bc == "periodic" and min(ext) < 2 * r + 1:
        pytest.skip("periodic grids need extents >= 2r+1")
    field, u0, _ = _case(dim, shape, r, ext, seed=500 + 10 * dim + r)
    for T in (1, 6):
        for arith in ("fma", "unfused"):
            ref = _oracle(u0, T, dim, shape, r, field, "jacobi", bc, 0.3, arith)
            got = _gpu(u0, T, dim, shape, r, field, "jacobi", bc, 0.3, arith)
            assert bits_equal(got, ref), (T, arith, first_diff(got, ref))


GS_CASES = [
    (1, "star", 1, (1000,), "constant"), (1, "star", 2, (301,), "constant"), (1, "star", 1, (77,), "periodic"),
    (2, "star", 1, (37, 130), "constant"), (2, "box", 1, (70, 131), "constant"), (2, "star", 2, (64, 65), "constant"),
    (2, "box", 2, (33, 70), "constant"), (2, "star", 1, (40, 33), "periodic"), (2, "star", 2, (30, 41), "periodic"),
    (2, "box", 1, (12, 13), "periodic"),
    (3, "star", 1, (9, 10, 21), "constant"), (3, "box", 1, (9, 10, 21), "constant"),
    (3, "star", 1, (10, 11, 12), "periodic"), (3, "star", 2, (10, 11, 12), "periodic"),
]


@pytest.mark.parametrize("dim,shape,r,ext,bc", GS_CASES)
@pytest.mark.parametrize("plan", [PLAIN, None])
def test_gs_field(dim, shape, r, ext, bc, plan):
    """None = the automatic plan: the wavefront (constant boundary) or the sweep DAG (periodic star)."""
    field, u0, _ = _case(dim, shape, r, ext, seed=600 + 10 * dim + r)
    for T in (1, 5, 33):
        for arith in ("fma", "unfused"):
            ref = _oracle(u0, T, dim, shape, r, field, "gs", bc, 0.3, arith)
            got = _gpu(u0, T, dim, shape, r, field, "gs", bc, 0.3, arith, plan=plan)
            assert bits_equal(got, ref), (T, arith, first_diff(got, ref))


def test_gs1d_wavefront_field_ragged_sweep_blocks():
    """1D wavefront with a field: T not a multiple of the 32 lanes, several sweep blocks."""
    field, u0, _ = _case(1, "star", 1, (4099,), seed=650)
    for T in (31, 32, 97):
        ref = _oracle(u0, T, 1, "star", 1, field, "gs", "constant", 0.0, "fma")
        got = _gpu(u0, T, 1, "star", 1, field, "gs", "constant", 0.0, "fma", plan=WAVE)
        assert bits_equal(got, ref), (T, first_diff(got, ref))


def test_uniform_field_equals_constant_weights():
    """A field repeating the constant weights at every point gives the constant-weight kernels' result."""
    import torch
    from paper_2010_04868_gb300 import stencil as S
    ext = (65, 130)
    w = inputs.normalized_weights(661, 9)
    u0 = torch.from_numpy(inputs.grid(662, ext)).cuda()
    field = torch.from_numpy(np.broadcast_to(np.asarray(w).reshape(9, 1, 1), (9,) + ext).copy()).cuda()
    for method in (0, 1):
        a = S.Stencil(2, 1, 1, list(w), method)
        b = S.Stencil(2, 1, 1, [0.0] * 9, method).set_field(field)
        ua, ub = u0.clone(), u0.clone()
        sa = torch.empty_like(ua) if method == 0 else None
        sb = torch.empty_like(ub) if method == 0 else None
        a.run(ua, 20, sa)
        b.run(ub, 20, sb)
        assert a.status() == 0 and b.status() == 0
        assert torch.equal(ua, ub)
        a.close()
        b.close()


def test_field_binding_errors_and_unbinding():
    import torch
    from paper_2010_04868_gb300 import stencil as S
    ext = (40, 50)
    w = inputs.normalized_weights(671, 5)
    field = torch.from_numpy(inputs.normalized_field(672, 5, ext)).cuda()
    u0 = torch.from_numpy(inputs.grid(673, ext)).cuda()
    st = S.Stencil(2, 0, 1, list(w), 0).set_field(field)
    # other extents: EINVAL while the field is bound
    other = torch.zeros((40, 51), dtype=torch.float64, device="cuda")
    with pytest.raises(S.StencilError) as e:
        st.run(other, 1, torch.empty_like(other))
    assert e.value.code == S.STENCIL_EINVAL
    # the temporally blocked kernel takes constant weights only
    st.set_plan(BLOCKED, 2, (0, 16, 64))
    u = u0.clone()
    with pytest.raises(S.StencilError) as e:
        st.run(u, 4, torch.empty_like(u))
    assert e.value.code == S.STENCIL_EUNSUPPORTED
    st.set_plan(0)
    # unbinding restores the constant weights
    st.set_field(None)
    u = u0.clone()
    st.run(u, 3, torch.empty_like(u))
    assert st.status() == 0
    ref = oracle.run(u0.cpu().numpy(), 3, dim=2, shape=0, r=1, weights=w)
    assert bits_equal(u.cpu().numpy(), ref)
    # a misaligned field pointer is rejected
    h = st.handle
    e3 = (ctypes.c_int64 * 3)(40, 50, 1)
    assert S.load().stencil_set_coeff_field(h, ctypes.c_void_p(field.data_ptr() + 4), e3) == S.STENCIL_EINVAL
    st.close()


def test_batch_with_field_problem_equals_separate_runs():
    """A problem with a field runs as its own launches inside a batch; results equal separate runs."""
    import torch
    from paper_2010_04868_gb300 import stencil as S
    ext = (70, 90)
    f = torch.from_numpy(inputs.normalized_field(681, 5, ext)).cuda()
    w = inputs.normalized_weights(682, 5)
    u0 = [torch.from_numpy(inputs.grid(683 + i, ext)).cuda() for i in range(3)]
    sts = [S.Stencil(2, 0, 1, list(w), 0).set_field(f), S.Stencil(2, 0, 1, list(w), 0),
           S.Stencil(2, 0, 1, [0.0] * 5, 1).set_field(f)]
    Ts = [7, 9, 5]
    us = [u.clone() for u in u0]
    scs = [torch.empty_like(us[0]), torch.empty_like(us[1]), None]
    grids = [st.grid(u, sc) for st, u, sc in zip(sts, us, scs)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):       # first call prepares and captures, second replays
        for u, v in zip(us, u0):
            u.copy_(v)
        S.stencil_run_batch([s.handle for s in sts], grids, Ts, stream)
        torch.cuda.synchronize()
        for st, u, v, T, meth in zip(sts, us, u0, Ts, ("jacobi", "jacobi", "gs")):
            assert st.status() == 0
            fld = f.cpu().numpy() if st is not sts[1] else None
            ref = oracle.run(v.cpu().numpy(), T, dim=2, shape=0, r=1, weights=w if fld is None else [0.0] * 5,
                             method=METHOD_ID[meth], field=fld)
            assert bits_equal(u.cpu().numpy(), ref)
    for st in sts:
        st.close()


def test_noalloc_with_field():
    import torch
    from paper_2010_04868_gb300 import stencil as S
    ext = (33, 47)
    f = torch.from_numpy(inputs.normalized_field(691, 9, ext)).cuda()
    u0 = inputs.grid(692, ext)
    st = S.Stencil(2, 1, 1, [0.0] * 9, 0).set_field(f)
    u = torch.from_numpy(u0).cuda()
    S.stencil_run_noalloc(st.handle, st.grid(u), 4, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st.status() == 0
    ref = oracle.run(u0, 4, dim=2, shape=1, r=1, weights=[0.0] * 9, field=f.cpu().numpy())
    assert bits_equal(u.cpu().numpy(), ref)
    st.close()


def test_jacobi2d_field_full_size():
    """The 4096^2 variable-coefficient 5-point Jacobi workload in its launch configuration, T cut to 3."""
    ext = (4096, 4096)
    field = inputs.normalized_field(inputs.SEED_BASE + 405, 5, ext)
    u0 = inputs.grid(inputs.SEED_BASE + 406, ext)
    ref = _oracle(u0, 3, 2, "star", 1, field, "jacobi", "constant", 0.0, "fma")
    got = _gpu(u0, 3, 2, "star", 1, field, "jacobi", "constant", 0.0, "fma")
    assert bits_equal(got, ref), first_diff(got, ref)


@pytest.mark.parametrize("ext", [(37, 132), (64, 64), (1, 8), (97, 36), (33, 68)])
@pytest.mark.parametrize("c", [0.0, 0.2])
def test_gs2d_rows_field_equals_oracle(ext, c):
    """The 2D Gauss-Seidel wavefront's default plan with a weight field on whole groups of four
    columns (rows as lanes, each lane loading its row's weights a step ahead): bit for bit."""
    field, u0, _ = _case(2, "star", 1, ext, seed=700 + ext[0])
    for T in (1, 5, 33):
        for arith in ("fma", "unfused"):
            ref = _oracle(u0, T, 2, "star", 1, field, "gs", "constant", c, arith)
            got = _gpu(u0, T, 2, "star", 1, field, "gs", "constant", c, arith, plan=WAVE)
            assert bits_equal(got, ref), (T, arith, first_diff(got, ref))


def test_gs2d_rows_field_full_size():
    """The 4096^2 field workload's grid (per-point weights), T cut to 12 for the serial oracle."""
    field, u0, _ = _case(2, "star", 1, (4096, 4096), seed=415)
    ref = _oracle(u0, 12, 2, "star", 1, field, "gs", "constant", 0.0, "fma")
    got = _gpu(u0, 12, 2, "star", 1, field, "gs", "constant", 0.0, "fma", plan=WAVE)
    assert bits_equal(got, ref), first_diff(got, ref)
