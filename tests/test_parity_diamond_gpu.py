"""Parity of the split-tiled (diamond) Jacobi kernel with the oracle, bit for bit.

The diamond plan tiles every used axis into A segments (trapezoids in
space-time) and B segments (inverted trapezoids), runs the 2^dim tile types of
a band as separate phases and works in place; in 1D, when every period fits
on the GPU at once, one persistent launch runs A and B of each period
together (neighbouring periods exchange edge values through flags). The cases cover one to many
periods per axis, ragged periods, band heights that the shortest period
forces down, T below, at and above the band height, radii 1..4, both
boundaries and both rounding modes.
"""
import ctypes

import numpy as np
import pytest

from helpers import bits_equal, case, first_diff, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

DIAMOND = 4

CASES = [
    # dim, shape, r, ext, H, periods (slowest first, padded to 3)
    (1, "star", 1, (2,), 4, (0, 0, 0)),
    (1, "star", 1, (37,), 4, (0, 0, 10)),
    (1, "star", 1, (4099,), 8, (0, 0, 256)),
    (1, "star", 1, (1000,), 32, (0, 0, 0)),
    (1, "star", 2, (3001,), 5, (0, 0, 97)),
    (1, "star", 3, (500,), 6, (0, 0, 64)),
    (1, "star", 4, (777,), 3, (0, 0, 100)),
    (1, "star", 1, (20000,), 8, (0, 0, 16)),       # 1250 periods: more than can be resident, phase launches
    (1, "star", 2, (9000,), 40, (0, 0, 0)),        # one period per SM: the concurrent kernel
    (2, "star", 1, (2, 3), 2, (0, 0, 0)),
    (2, "star", 1, (130, 258), 4, (0, 40, 64)),
    (2, "star", 1, (131, 257), 6, (0, 0, 0)),
    (2, "box", 1, (200, 96), 3, (0, 48, 30)),
    (2, "box", 1, (61, 77), 5, (0, 20, 13)),
    (2, "star", 2, (64, 66), 2, (0, 16, 32)),
    (2, "box", 2, (40, 50), 2, (0, 16, 16)),
    (3, "star", 1, (20, 18, 40), 2, (0, 0, 0)),
    (3, "box", 1, (17, 9, 34), 2, (8, 4, 16)),
    (3, "star", 1, (33, 29, 31), 3, (12, 10, 14)),
    (3, "star", 2, (9, 12, 20), 1, (4, 4, 8)),
]


@pytest.mark.parametrize("dim,shape,r,ext,H,periods", CASES)
@pytest.mark.parametrize("bc,c", [("constant", 0.0), ("constant", 0.7), ("periodic", 0.0)])
def test_jacobi_diamond(dim, shape, r, ext, H, periods, bc, c):
    if bc == "periodic" and min(ext) < 2 * r + 1:
        pytest.skip("periodic needs ext >= 2r+1")
    if min(ext) < 2 * r:
        pytest.skip("an axis shorter than 2r points cannot be split-tiled")
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r + 5)
    for T in (1, H - 1, H, H + 1, 3 * H + 2):
        if T < 1:
            continue
        for arith in ("fma", "unfused"):
            ref = oracle_run(u0, T, dim, shape, r, w, "jacobi", bc, c, arith)
            got = gpu_run(u0, T, dim, shape, r, w, "jacobi", bc, c, arith, plan=DIAMOND, tb=H, tile=periods,
                          use_scratch=False)
            assert bits_equal(got, ref), (T, arith, first_diff(got, ref))


def test_axis_too_short_is_unsupported():
    import torch
    from paper_2010_04868_gb300 import stencil as S
    st = S.Stencil(1, 0, 2, [0.1, 0.2, 0.4, 0.2, 0.1], S.STENCIL_JACOBI)
    st.set_plan(DIAMOND, 4, (0, 0, 0))
    u = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(S.StencilError) as e:
        st.run(u, 5)
    assert e.value.code == S.STENCIL_EUNSUPPORTED
    st.close()


def test_heat1d_full_size_diamond_equals_oracle():
    """The 1D heat workload at full size (N = 65536, T = 256, weights 1/4, 1/2, 1/4, zero halo)."""
    from paper_2010_04868_gb300 import inputs
    u0 = inputs.grid(inputs.SEED_BASE + 1, (65536,))
    w = [0.25, 0.5, 0.25]
    ref = oracle_run(u0, 256, 1, "star", 1, w, "jacobi", "constant", 0.0, "fma")
    for H, P in ((64, 0), (32, 216), (128, 431), (100, 1000)):
        got = gpu_run(u0, 256, 1, "star", 1, w, "jacobi", "constant", 0.0, "fma", plan=DIAMOND, tb=H,
                      tile=(0, 0, P), use_scratch=False)
        assert bits_equal(got, ref), (H, P, first_diff(got, ref))


@pytest.mark.parametrize("shape", ["star", "box"])
def test_jacobi2d_full_size_diamond_equals_plain(shape):
    """4096^2 with normalized weights: the diamond plan equals the plain kernel (itself pinned to the oracle)."""
    w, u0 = case(2, shape, 1, (4096, 4096), seed=77)
    T = 30
    plain = gpu_run(u0, T, 2, shape, 1, w, "jacobi", "constant", 0.0, "fma", plan=1)
    for H, P in ((12, (0, 96, 96)), (8, (0, 64, 128))):
        got = gpu_run(u0, T, 2, shape, 1, w, "jacobi", "constant", 0.0, "fma", plan=DIAMOND, tb=H, tile=P,
                      use_scratch=False)
        assert bits_equal(got, plain), (H, P, first_diff(got, plain))
    # sampled points against the oracle: after T steps a point depends only on points within T of it
    # (Chebyshev distance), so the oracle run on the (2T+1)^2 window centred on it gives its exact value;
    # the window at a corner is flush with two grid edges and gives the exact corner block
    rng = np.random.default_rng(5)
    for i, j in [tuple(int(v) for v in rng.integers(T, 4096 - T, 2)) for _ in range(4)]:
        win = u0[i - T:i + T + 1, j - T:j + T + 1].copy()
        ref = oracle_run(win, T, 2, shape, 1, w, "jacobi", "constant", 0.0, "fma")
        assert bits_equal(got[i, j], ref[T, T]), (i, j)
    win = u0[:2 * T + 1, :2 * T + 1].copy()
    ref = oracle_run(win, T, 2, shape, 1, w, "jacobi", "constant", 0.0, "fma")
    assert bits_equal(got[:T + 1, :T + 1], ref[:T + 1, :T + 1])


def test_periodic_3d_diamond_equals_plain():
    w, u0 = case(3, "star", 1, (96, 80, 128), seed=21)
    T = 9
    plain = gpu_run(u0, T, 3, "star", 1, w, "jacobi", "periodic", 0.0, "fma", plan=1)
    got = gpu_run(u0, T, 3, "star", 1, w, "jacobi", "periodic", 0.0, "fma", plan=DIAMOND, tb=4, tile=(24, 20, 32),
                  use_scratch=False)
    assert bits_equal(got, plain), first_diff(got, plain)


@pytest.mark.parametrize("dim,ext,H,periods", [(2, (300, 257), 4, (0, 64, 64)), (1, (30011,), 40, (0, 0, 0))])
def test_diamond_run_replays_in_a_cuda_graph(dim, ext, H, periods):
    """After one run has sized the workspace, a run captured into a CUDA graph replays to the same grid
    (2D: the phase launches; 1D: the concurrent kernel with its flag reset)."""
    import torch
    from paper_2010_04868_gb300 import stencil as S
    w, u0 = case(dim, "star", 1, ext, seed=3)
    T = 11 if dim == 2 else 97
    ref = oracle_run(u0, T, dim, "star", 1, w, "jacobi", "constant", 0.0, "fma")
    st = S.Stencil(dim, 0, 1, list(w), S.STENCIL_JACOBI)
    st.set_plan(DIAMOND, H, periods)
    u = torch.from_numpy(u0.copy()).cuda()
    st.run(u, T)
    assert st.status() == 0
    assert bits_equal(u.cpu().numpy(), ref)
    u.copy_(torch.from_numpy(u0))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            st.run(u, T, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        u.copy_(torch.from_numpy(u0))
        graph.replay()
        torch.cuda.synchronize()
        assert bits_equal(u.cpu().numpy(), ref)
    st.close()


@pytest.mark.parametrize("bc,unit", [(0, 5), (0, 0), (1, 77)])
def test_concurrent_1d_stalled_period_times_out_without_hanging(bc, unit):
    """A period of the concurrent 1D kernel that never publishes its edges makes its neighbours'
    bounded waits expire: the launch finishes, stencil_status() reports ETIMEOUT, and the next
    run on the same handle is correct again."""
    import torch
    from paper_2010_04868_gb300 import stencil as S
    w, u0 = case(1, "star", 2, (9000,), seed=41)
    T = 90
    st = S.Stencil(1, 0, 2, list(w), S.STENCIL_JACOBI, bc).set_plan(DIAMOND, 40, (0, 0, 0))
    u = torch.from_numpy(u0.copy()).cuda()
    S.stencil_debug_inject_stall(st.handle, unit, 20000)
    st.run(u, T)
    assert st.status() == S.STENCIL_ETIMEOUT
    u.copy_(torch.from_numpy(u0))
    st.run(u, T)
    assert st.status() == 0
    ref = oracle_run(u0, T, 1, "star", 2, w, "jacobi", "periodic" if bc else "constant", 0.0, "fma")
    assert bits_equal(u.cpu().numpy(), ref), first_diff(u.cpu().numpy(), ref)
    st.close()
