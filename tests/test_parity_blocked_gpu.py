"""Parity of the temporally blocked Jacobi kernel with the oracle, bit for bit."""
import numpy as np
import pytest

from helpers import bits_equal, case, first_diff, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

BLOCKED = 2

CASES = [
    # dim, shape, r, ext, tb, tile
    (1, "star", 1, (1,), 4, (0, 0, 0)),
    (1, "star", 1, (4099,), 8, (0, 0, 256)),
    (1, "star", 1, (1000,), 32, (0, 0, 0)),
    (1, "star", 2, (3001,), 5, (0, 0, 512)),
    (1, "star", 4, (777,), 3, (0, 0, 100)),
    (2, "star", 1, (1, 2), 2, (0, 0, 0)),
    (2, "star", 1, (130, 258), 2, (0, 64, 64)),
    (2, "star", 1, (131, 257), 4, (0, 32, 64)),     # odd inner extent: staged without TMA
    (2, "box", 1, (200, 96), 3, (0, 48, 96)),
    (2, "star", 2, (64, 66), 2, (0, 16, 32)),
    (2, "box", 2, (40, 50), 2, (0, 16, 16)),
    (3, "star", 1, (20, 18, 40), 2, (0, 0, 0)),
    (3, "box", 1, (17, 9, 34), 2, (4, 8, 16)),
    (3, "star", 2, (9, 12, 20), 1, (4, 4, 8)),
]


@pytest.mark.parametrize("dim,shape,r,ext,tb,tile", CASES)
@pytest.mark.parametrize("bc,c", [("constant", 0.0), ("constant", 0.7), ("periodic", 0.0)])
def test_jacobi_blocked(dim, shape, r, ext, tb, tile, bc, c):
    if bc == "periodic" and min(ext) < 2 * r + 1:
        pytest.skip("periodic needs ext >= 2r+1")
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r + 2)
    for T in (1, tb - 1, tb, tb + 1, 3 * tb + 2):
        if T < 1:
            continue
        for arith in ("fma", "unfused"):
            ref = oracle_run(u0, T, dim, shape, r, w, "jacobi", bc, c, arith)
            got = gpu_run(u0, T, dim, shape, r, w, "jacobi", bc, c, arith, plan=BLOCKED, tb=tb, tile=tile)
            assert bits_equal(got, ref), (T, arith, first_diff(got, ref))


def test_heat1d_full_size_blocked_equals_oracle():
    """The 1D heat workload at full size (N = 65536, T = 256, weights 1/4, 1/2, 1/4, zero halo)."""
    from paper_2010_04868_gb300 import inputs
    u0 = inputs.grid(inputs.SEED_BASE + 1, (65536,))
    w = [0.25, 0.5, 0.25]
    ref = oracle_run(u0, 256, 1, "star", 1, w, "jacobi", "constant", 0.0, "fma")
    for tb in (16, 32, 64):
        got = gpu_run(u0, 256, 1, "star", 1, w, "jacobi", "constant", 0.0, "fma", plan=BLOCKED, tb=tb)
        assert bits_equal(got, ref), (tb, first_diff(got, ref))
