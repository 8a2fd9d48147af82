"""Parity of the plain kernels with the oracle, bit for bit, through the C ABI."""
import numpy as np
import pytest

from helpers import bits_equal, case, first_diff, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

PLAIN = 1

JACOBI_CASES = [
    # dim, shape, r, ext
    (1, "star", 1, (1,)), (1, "star", 1, (37,)), (1, "star", 1, (4099,)), (1, "star", 2, (1000,)),
    (1, "star", 3, (301,)), (1, "star", 4, (97,)),
    (2, "star", 1, (1, 1)), (2, "star", 1, (37, 130)), (2, "box", 1, (257, 131)), (2, "star", 2, (64, 65)),
    (2, "box", 2, (33, 70)), (2, "star", 3, (20, 41)),
    (3, "star", 1, (5, 6, 7)), (3, "box", 1, (33, 17, 40)), (3, "star", 2, (9, 10, 33)), (3, "box", 2, (7, 8, 9)),
]


@pytest.mark.parametrize("dim,shape,r,ext", JACOBI_CASES)
@pytest.mark.parametrize("bc,c", [("constant", 0.0), ("constant", 0.3), ("periodic", 0.0)])
@pytest.mark.parametrize("arith", ["fma", "unfused"])
def test_jacobi_plain(dim, shape, r, ext, bc, c, arith):
    if bc == "periodic" and min(ext) < 2 * r + 1:
        pytest.skip("periodic needs ext >= 2r+1")
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r)
    for T in (1, 2, 5):
        ref = oracle_run(u0, T, dim, shape, r, w, "jacobi", bc, c, arith)
        got = gpu_run(u0, T, dim, shape, r, w, "jacobi", bc, c, arith, plan=PLAIN)
        assert bits_equal(got, ref), (T, first_diff(got, ref))


GS_CASES = [
    (1, "star", 1, (1,)), (1, "star", 1, (37,)), (1, "star", 1, (2051,)), (1, "star", 2, (300,)), (1, "star", 4, (50,)),
    (2, "star", 1, (1, 1)), (2, "star", 1, (37, 130)), (2, "box", 1, (70, 131)), (2, "star", 2, (64, 65)),
    (2, "box", 2, (33, 70)), (2, "star", 3, (12, 21)),
    (3, "star", 1, (5, 6, 7)), (3, "box", 1, (20, 17, 40)), (3, "star", 2, (9, 10, 33)), (3, "box", 2, (6, 7, 8)),
]


@pytest.mark.parametrize("dim,shape,r,ext", GS_CASES)
@pytest.mark.parametrize("bc,c", [("constant", 0.0), ("constant", 0.3), ("periodic", 0.0)])
@pytest.mark.parametrize("arith", ["fma", "unfused"])
def test_gs_plain(dim, shape, r, ext, bc, c, arith):
    if bc == "periodic" and min(ext) < 2 * r + 1:
        pytest.skip("periodic needs ext >= 2r+1")
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r + 5)
    for T in (1, 3):
        ref = oracle_run(u0, T, dim, shape, r, w, "gs", bc, c, arith)
        got = gpu_run(u0, T, dim, shape, r, w, "gs", bc, c, arith, plan=PLAIN)
        assert bits_equal(got, ref), (T, first_diff(got, ref))


def test_jacobi_without_scratch_and_odd_T():
    w, u0 = case(2, "star", 1, (100, 77), seed=3)
    for T in (0, 1, 4, 7):
        ref = oracle_run(u0, T, 2, "star", 1, w, "jacobi", "constant", 0.0, "fma")
        got = gpu_run(u0, T, 2, "star", 1, w, "jacobi", "constant", 0.0, "fma", plan=PLAIN, use_scratch=False)
        assert bits_equal(got, ref)


def test_split_runs_equal_one_run():
    """run(T1) then run(T2) equals run(T1+T2): the grid is the whole state (checkpoint/resume)."""
    import torch
    from paper_2010_04868_gb300 import stencil as S
    w, u0 = case(2, "box", 1, (65, 90), seed=4)
    for method in (S.STENCIL_JACOBI, S.STENCIL_GAUSS_SEIDEL):
        st = S.Stencil(2, S.STENCIL_BOX, 1, list(w), method)
        a = torch.from_numpy(u0.copy()).cuda()
        b = torch.from_numpy(u0.copy()).cuda()
        st.run(a, 7)
        st.run(b, 3)
        st.run(b, 4)
        assert torch.equal(a, b)
        st.close()


def test_argument_errors():
    import torch
    from paper_2010_04868_gb300 import stencil as S
    with pytest.raises(S.StencilError):
        S.Stencil(2, 0, 1, [1.0] * 4)                        # K mismatch
    with pytest.raises(S.StencilError):
        S.Stencil(4, 0, 1, [1.0] * 9)                        # dim > 3
    st = S.Stencil(1, 0, 2, [0.2] * 5, boundary=S.STENCIL_BC_PERIODIC)
    u = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(S.StencilError) as e:
        st.run(u, 1)                                         # periodic needs ext >= 2r+1
    assert e.value.code == S.STENCIL_EINVAL
    with pytest.raises(S.StencilError):
        st.run(torch.zeros(8, dtype=torch.float64, device="cuda"), -1)
    st.close()


@pytest.mark.parametrize("dim,ext,kernel,tb,T", [(2, (300, 257), 1, 0, 9), (3, (40, 33, 70), 1, 0, 6),
                                                 (1, (20000,), 2, 8, 37), (2, (130, 515), 2, 4, 11)])
def test_programmatic_launches_replay_in_a_cuda_graph(dim, ext, kernel, tb, T):
    """Plain steps and blocked passes are launched with programmatic stream serialization; a run captured
    into a CUDA graph (the launches become programmatic edges) replays to the oracle's grid, after
    other work on the same stream."""
    import torch
    from paper_2010_04868_gb300 import stencil as S
    w, u0 = case(dim, "star", 1, ext, seed=dim + 17)
    ref = oracle_run(u0, T, dim, "star", 1, w, "jacobi", "constant", 0.25, "fma")
    st = S.Stencil(dim, 0, 1, list(w), S.STENCIL_JACOBI, S.STENCIL_BC_CONSTANT, 0.25)
    st.set_plan(kernel, tb)
    u = torch.from_numpy(u0.copy()).cuda()
    scratch = torch.empty_like(u)
    src = torch.from_numpy(u0.copy()).cuda()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            u.copy_(src)        # a kernel of another library right before the first programmatic launch
            st.run(u, T, scratch=scratch, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        u.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert st.status() == 0
        got = u.cpu().numpy()
        assert bits_equal(got, ref), first_diff(got, ref)
    st.close()


@pytest.mark.parametrize("shape,k", [("star", 5), ("box", 9)])
def test_jacobi2d_full_size_plain_equals_oracle_whole_grid(shape, k):
    """The 4096^2 Jacobi workload's seeded grid and weights, plain per-step kernel in its launch configuration,
    T = 3, against the oracle on every point."""
    from paper_2010_04868_gb300 import inputs
    ext = (4096, 4096)
    w = inputs.normalized_weights(inputs.SEED_BASE + 100 + k, k)
    u0 = inputs.grid(inputs.SEED_BASE + 2, ext)
    ref = oracle_run(u0, 3, 2, shape, 1, w, "jacobi", "constant", 0.0, "fma")
    got = gpu_run(u0, 3, 2, shape, 1, w, "jacobi", "constant", 0.0, "fma", plan=1)
    assert bits_equal(got, ref), first_diff(got, ref)


@pytest.mark.parametrize("dim,shape,ext,rb", [(2, "star", (37, 130), 2), (2, "box", (257, 131), 2),
                                              (2, "star", (66, 65), 4), (3, "star", (33, 17, 40), 1),
                                              (3, "box", (9, 10, 37), 1), (3, "star", (10, 13, 35), 2)])
@pytest.mark.parametrize("bc,c", [("constant", 0.3), ("periodic", 0.0)])
def test_jacobi_plain_points_per_thread(dim, shape, ext, rb, bc, c):
    """The plain step with the points per thread a plain plan fixes (tile[2])."""
    w, u0 = case(dim, shape, 1, ext, seed=dim * 13 + rb)
    for arith in ("fma", "unfused"):
        ref = oracle_run(u0, 5, dim, shape, 1, w, "jacobi", bc, c, arith)
        got = gpu_run(u0, 5, dim, shape, 1, w, "jacobi", bc, c, arith, plan=PLAIN, tile=(0, 0, rb))
        assert bits_equal(got, ref), (arith, first_diff(got, ref))
