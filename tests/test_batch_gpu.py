"""Batched persistent execution: every problem's result equals its own run and the oracle, bit for bit."""
import numpy as np
import pytest

from helpers import BC_ID, METHOD_ID, SHAPE_ID, bits_equal, case, first_diff, oracle_run

pytestmark = pytest.mark.gpu

PLAIN, BLOCKED, WAVE = 1, 2, 3

MIX = [
    # dim, shape, r, ext, method, bc, c, T, plan (kernel, tb, tile)
    (1, "star", 1, (5000,), "jacobi", "constant", 0.0, 37, (BLOCKED, 16, (0, 0, 256))),
    (1, "star", 2, (777,), "jacobi", "periodic", 0.0, 9, (PLAIN, 0, (0, 0, 0))),
    (2, "star", 1, (130, 97), "jacobi", "constant", 0.3, 11, (PLAIN, 0, (0, 0, 0))),
    (2, "box", 1, (64, 200), "jacobi", "constant", 0.0, 7, (BLOCKED, 3, (0, 32, 64))),
    (3, "star", 1, (20, 21, 22), "jacobi", "periodic", 0.0, 6, (PLAIN, 0, (0, 0, 0))),
    (3, "box", 1, (17, 18, 30), "jacobi", "constant", 0.5, 5, (BLOCKED, 2, (8, 8, 16))),
    (2, "star", 1, (70, 81), "gs", "periodic", 0.0, 4, (PLAIN, 0, (0, 0, 0))),
    (2, "box", 1, (40, 90), "gs", "constant", 0.2, 3, (PLAIN, 0, (0, 0, 0))),
    (3, "star", 1, (19, 20, 21), "gs", "periodic", 0.0, 3, (PLAIN, 0, (0, 0, 0))),
    (3, "box", 1, (9, 10, 11), "gs", "constant", 0.0, 2, (PLAIN, 0, (0, 0, 0))),
    (1, "star", 1, (300,), "gs", "periodic", 0.0, 3, (PLAIN, 0, (0, 0, 0))),
    (2, "star", 1, (50, 60), "gs", "constant", 0.1, 40, (WAVE, 0, (0, 0, 0))),
    (1, "star", 1, (3000,), "gs", "constant", 0.0, 45, (WAVE, 0, (0, 0, 0))),
    (2, "box", 1, (33, 44), "jacobi", "constant", 0.0, 0, (PLAIN, 0, (0, 0, 0))),     # T = 0: untouched
]


def _setup(mix, seed0=0):
    import torch
    from paper_2010_04868_gb300 import stencil as S
    sts, grids, Ts, tensors, refs = [], [], [], [], []
    for n, (dim, shape, r, ext, method, bc, c, T, plan) in enumerate(mix):
        w, u0 = case(dim, shape, r, ext, seed=seed0 + n + 1)
        st = S.Stencil(dim, SHAPE_ID[shape], r, list(w), METHOD_ID[method], BC_ID[bc], c)
        st.set_plan(*plan)
        u = torch.from_numpy(u0.copy()).cuda()
        sc = torch.empty_like(u) if method == "jacobi" else None
        sts.append(st)
        grids.append(st.grid(u, sc))
        Ts.append(T)
        tensors.append((u, sc, u0))
        refs.append(oracle_run(u0, T, dim, shape, r, w, method, bc, c, "fma"))
    return sts, grids, Ts, tensors, refs


def test_batch_mixed_equals_oracle_and_replays():
    import ctypes
    import torch
    from paper_2010_04868_gb300 import stencil as S
    sts, grids, Ts, tensors, refs = _setup(MIX)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for rep in range(3):                                   # capture, then replay the cached graph twice
        for (u, sc, u0) in tensors:
            u.copy_(torch.from_numpy(u0))
        S.stencil_run_batch([s.handle for s in sts], grids, Ts, stream)
        torch.cuda.synchronize()
        for n, (st, (u, _, _), ref) in enumerate(zip(sts, tensors, refs)):
            assert st.status() == 0
            got = u.cpu().numpy()
            assert bits_equal(got, ref), (rep, n, MIX[n], first_diff(got, ref))
    for st in sts:
        st.close()


def test_batch_inside_caller_capture():
    """A batch enqueued on a stream the caller is already capturing runs correctly when the caller replays."""
    import ctypes
    import torch
    from paper_2010_04868_gb300 import stencil as S
    mix = [m for m in MIX if m[8][0] != WAVE][:6]
    sts, grids, Ts, tensors, refs = _setup(mix, seed0=20)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):                        # first run outside capture prepares the batch
        S.stencil_run_batch([x.handle for x in sts], grids, Ts, ctypes.c_void_p(s.cuda_stream))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        S.stencil_run_batch([x.handle for x in sts], grids, Ts, ctypes.c_void_p(s.cuda_stream))
    for rep in range(2):
        for (u, sc, u0) in tensors:
            u.copy_(torch.from_numpy(u0))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        for n, ((u, _, _), ref) in enumerate(zip(tensors, refs)):
            assert bits_equal(u.cpu().numpy(), ref), (rep, n)
    for st in sts:
        st.close()


def test_new_batch_inside_caller_capture_is_refused():
    import ctypes
    import torch
    from paper_2010_04868_gb300 import stencil as S
    sts, grids, Ts, tensors, refs = _setup(MIX[2:3], seed0=40)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(S.StencilError) as e:
        with torch.cuda.graph(g, stream=s):
            S.stencil_run_batch([x.handle for x in sts], grids, Ts, ctypes.c_void_p(s.cuda_stream))
    assert e.value.code == S.STENCIL_EUNSUPPORTED
    for st in sts:
        st.close()


def test_batch_periodic_3d_full_size_equals_solo():
    """The 512^3 periodic mix (Jacobi 7P, Jacobi 27P, Gauss-Seidel 7P) at T = 100 in one batch vs separate runs."""
    import ctypes
    import torch
    from paper_2010_04868_gb300 import inputs
    from paper_2010_04868_gb300 import stencil as S
    ext = (512, 512, 512)
    specs = [(0, 7, S.STENCIL_JACOBI), (1, 27, S.STENCIL_JACOBI), (0, 7, S.STENCIL_GAUSS_SEIDEL)]
    u0 = torch.from_numpy(inputs.grid(inputs.SEED_BASE + 5, ext)).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sts, grids, us, scs = [], [], [], []
    for shape, k, method in specs:
        st = S.Stencil(3, shape, 1, list(inputs.normalized_weights(inputs.SEED_BASE + 200 + k + method, k)), method,
                       S.STENCIL_BC_PERIODIC)
        u = u0.clone()
        sc = torch.empty_like(u) if method == S.STENCIL_JACOBI else None
        sts.append(st)
        us.append(u)
        scs.append(sc)
        grids.append(st.grid(u, sc))
    S.stencil_run_batch([s.handle for s in sts], grids, [100, 100, 100], stream)
    torch.cuda.synchronize()
    for st, u, sc in zip(sts, us, scs):
        assert st.status() == 0
        v = u0.clone()
        st.set_plan(PLAIN)
        st.run(v, 100, torch.empty_like(v) if sc is not None else None)
        torch.cuda.synchronize()
        assert torch.equal(u, v)
        st.close()


def test_batch_periodic_3d_full_size_equals_oracle():
    """The 512^3 periodic mix (Jacobi 7P, Jacobi 27P, Gauss-Seidel 7P) in one batch at T = 2, in the batch's
    launch configuration, against the oracle on the whole grid, bit for bit."""
    import ctypes
    import torch
    import oracle
    from paper_2010_04868_gb300 import inputs
    from paper_2010_04868_gb300 import stencil as S
    ext = (512, 512, 512)
    T = 2
    specs = [(0, 7, S.STENCIL_JACOBI), (1, 27, S.STENCIL_JACOBI), (0, 7, S.STENCIL_GAUSS_SEIDEL)]
    u0h = inputs.grid(inputs.SEED_BASE + 6, ext)
    u0 = torch.from_numpy(u0h).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sts, grids, us, scs, ws = [], [], [], [], []
    for shape, k, method in specs:
        w = list(inputs.normalized_weights(inputs.SEED_BASE + 210 + k + method, k))
        st = S.Stencil(3, shape, 1, w, method, S.STENCIL_BC_PERIODIC)
        u = u0.clone()
        sc = torch.empty_like(u) if method == S.STENCIL_JACOBI else None
        sts.append(st)
        us.append(u)
        scs.append(sc)
        ws.append(w)
        grids.append(st.grid(u, sc))
    S.stencil_run_batch([s.handle for s in sts], grids, [T] * 3, stream)
    torch.cuda.synchronize()
    for st, u, w, (shape, k, method) in zip(sts, us, ws, specs):
        assert st.status() == 0
        ref = oracle.run(u0h, T, dim=3, shape=shape, r=1, weights=w, method=method, bc=1)
        got = u.cpu().numpy()
        assert bits_equal(got, ref), first_diff(got, ref)
        st.close()
