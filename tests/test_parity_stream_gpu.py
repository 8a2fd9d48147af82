"""Parity of the streaming temporally blocked Jacobi kernel (plan STREAM) with the oracle, bit for bit."""
import numpy as np
import pytest

from helpers import bits_equal, case, first_diff, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

STREAM = 5

CASES = [
    # dim, shape, r, ext, tb, tile (chunk Z, staged rows W1 (3D), staged columns W2)
    (2, "star", 1, (1, 2), 2, (0, 0, 0)),
    (2, "star", 1, (37, 70), 2, (0, 0, 32)),
    (2, "star", 1, (130, 258), 2, (0, 0, 0)),
    (2, "star", 1, (131, 257), 4, (16, 0, 64)),     # odd row pitch: staged with cp.async, not TMA
    (2, "box", 1, (200, 96), 3, (9, 0, 64)),
    (2, "box", 1, (301, 500), 1, (0, 0, 128)),
    (2, "star", 2, (64, 66), 2, (0, 0, 64)),
    (2, "box", 2, (40, 50), 1, (5, 0, 32)),
    (3, "star", 1, (20, 18, 40), 2, (0, 0, 0)),
    (3, "box", 1, (17, 9, 34), 2, (4, 8, 32)),
    (3, "star", 1, (9, 33, 70), 1, (3, 0, 64)),
    (3, "box", 1, (5, 6, 7), 1, (0, 0, 0)),
]


@pytest.mark.parametrize("dim,shape,r,ext,tb,tile", CASES)
@pytest.mark.parametrize("bc,c", [("constant", 0.0), ("constant", 0.7), ("periodic", 0.0)])
def test_jacobi_stream(dim, shape, r, ext, tb, tile, bc, c):
    if bc == "periodic" and min(ext) < 2 * r + 1:
        pytest.skip("periodic needs ext >= 2r+1")
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r + 5)
    for T in (1, tb, tb + 1, 3 * tb + 2):
        for arith in ("fma", "unfused"):
            ref = oracle_run(u0, T, dim, shape, r, w, "jacobi", bc, c, arith)
            got = gpu_run(u0, T, dim, shape, r, w, "jacobi", bc, c, arith, plan=STREAM, tb=tb, tile=tile)
            assert bits_equal(got, ref), (T, arith, first_diff(got, ref))


@pytest.mark.parametrize("shape,k,tb", [("star", 5, 2), ("star", 5, 4), ("box", 9, 2), ("box", 9, 3)])
def test_jacobi2d_full_size_stream_equals_oracle(shape, k, tb):
    """The 4096^2 Jacobi workload's seeded grid and weights in the stream plan's default launch
    geometry, against the oracle on every point (T = 2 T_b + 1: two passes and a plain step)."""
    from paper_2010_04868_gb300 import inputs
    ext = (4096, 4096)
    w = inputs.normalized_weights(inputs.SEED_BASE + 100 + k, k)
    u0 = inputs.grid(inputs.SEED_BASE + 2, ext)
    T = 2 * tb + 1
    ref = oracle_run(u0, T, 2, shape, 1, w, "jacobi", "constant", 0.0, "fma")
    got = gpu_run(u0, T, 2, shape, 1, w, "jacobi", "constant", 0.0, "fma", plan=STREAM, tb=tb)
    assert bits_equal(got, ref), first_diff(got, ref)


@pytest.mark.parametrize("shape,k,tb", [("star", 7, 1), ("star", 7, 2), ("box", 27, 1)])
def test_jacobi3d_full_size_periodic_stream_equals_oracle(shape, k, tb):
    """512^3 periodic (the 3D workloads' size and boundary), T = 2, against the oracle on every point."""
    from paper_2010_04868_gb300 import inputs
    ext = (512, 512, 512)
    w = inputs.normalized_weights(inputs.SEED_BASE + 207 + k, k)
    u0 = inputs.grid(inputs.SEED_BASE + 7, ext)
    ref = oracle_run(u0, 2, 3, shape, 1, w, "jacobi", "periodic", 0.0, "fma")
    got = gpu_run(u0, 2, 3, shape, 1, w, "jacobi", "periodic", 0.0, "fma", plan=STREAM, tb=tb)
    assert bits_equal(got, ref), first_diff(got, ref)


def test_stream_plan_refused_for_gauss_seidel_and_1d():
    from paper_2010_04868_gb300 import stencil as S
    gs = S.Stencil(2, 0, 1, [0.2] * 5, S.STENCIL_GAUSS_SEIDEL)
    with pytest.raises(S.StencilError):
        gs.set_plan(STREAM, 2)
    gs.close()
    import torch
    j1 = S.Stencil(1, 0, 1, [0.25, 0.5, 0.25], S.STENCIL_JACOBI).set_plan(STREAM, 2)
    u = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(S.StencilError) as e:
        j1.run(u, 3, torch.empty_like(u))
    assert e.value.code == S.STENCIL_EUNSUPPORTED
    j1.close()
