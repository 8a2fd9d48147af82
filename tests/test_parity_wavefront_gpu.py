"""Parity of the time-skewed wavefront Gauss-Seidel kernel with the oracle, bit for bit."""
import ctypes

import numpy as np
import pytest

from helpers import bits_equal, case, first_diff, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

WAVE = 3
PLAIN = 1

CASES_1D = [((1,), 1), ((37,), 1), ((1000,), 1), ((4099,), 1), ((300,), 2), ((101,), 3), ((64,), 4), ((3,), 1)]


@pytest.mark.parametrize("ext,r", CASES_1D)
@pytest.mark.parametrize("c", [0.0, 0.4])
def test_gs1d_wavefront(ext, r, c):
    w, u0 = case(1, "star", r, ext, seed=r + 60)
    for T in (1, 5, 31, 32, 33, 64, 97):
        for arith in ("fma", "unfused"):
            ref = oracle_run(u0, T, 1, "star", r, w, "gs", "constant", c, arith)
            got = gpu_run(u0, T, 1, "star", r, w, "gs", "constant", c, arith, plan=WAVE)
            assert bits_equal(got, ref), (T, arith, first_diff(got, ref))


CASES_ND = [
    (2, "star", 1, (1, 1)), (2, "star", 1, (37, 130)), (2, "star", 1, (130, 37)), (2, "box", 1, (70, 131)),
    (2, "star", 2, (64, 65)), (2, "box", 2, (33, 70)),
    (3, "star", 1, (5, 6, 7)), (3, "star", 1, (20, 17, 40)), (3, "box", 1, (9, 10, 21)),
]


@pytest.mark.parametrize("dim,shape,r,ext", CASES_ND)
@pytest.mark.parametrize("c", [0.0, 0.4])
def test_gs_nd_wavefront(dim, shape, r, ext, c):
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + r + 70)
    for T in (1, 7, 32, 45):
        for arith in ("fma", "unfused"):
            ref = oracle_run(u0, T, dim, shape, r, w, "gs", "constant", c, arith)
            got = gpu_run(u0, T, dim, shape, r, w, "gs", "constant", c, arith, plan=WAVE)
            assert bits_equal(got, ref), (T, arith, first_diff(got, ref))


def test_gs2d_full_size_wavefront_equals_oracle():
    """The 4096^2 Gauss-Seidel 5-point workload in its launch configuration, T cut to 24 for the serial oracle."""
    from paper_2010_04868_gb300 import inputs
    u0 = inputs.grid(inputs.SEED_BASE + 3, (4096, 4096))
    w = inputs.normalized_weights(inputs.SEED_BASE + 105, 5)
    ref = oracle_run(u0, 24, 2, "star", 1, w, "gs", "constant", 0.0, "fma")
    got = gpu_run(u0, 24, 2, "star", 1, w, "gs", "constant", 0.0, "fma", plan=WAVE)
    assert bits_equal(got, ref), first_diff(got, ref)


def test_gs2d_full_size_full_T_wavefront_equals_plain():
    """Full 4096^2 x 200 sweeps: wavefront and plain sweep kernels agree bit for bit."""
    from paper_2010_04868_gb300 import inputs
    u0 = inputs.grid(inputs.SEED_BASE + 3, (4096, 4096))
    w = inputs.normalized_weights(inputs.SEED_BASE + 105, 5)
    a = gpu_run(u0, 200, 2, "star", 1, w, "gs", "constant", 0.0, "fma", plan=WAVE)
    b = gpu_run(u0, 200, 2, "star", 1, w, "gs", "constant", 0.0, "fma", plan=PLAIN)
    assert bits_equal(a, b), first_diff(a, b)


def test_gs1d_long_wavefront_equals_oracle():
    """The 1D Gauss-Seidel workload at its full N = 2^24, T cut to 40 for the serial oracle."""
    from paper_2010_04868_gb300 import inputs
    u0 = inputs.grid(inputs.SEED_BASE + 4, (1 << 24,))
    w = inputs.normalized_weights(inputs.SEED_BASE + 103, 3)
    ref = oracle_run(u0, 40, 1, "star", 1, w, "gs", "constant", 0.0, "fma")
    got = gpu_run(u0, 40, 1, "star", 1, w, "gs", "constant", 0.0, "fma", plan=WAVE)
    assert bits_equal(got, ref), first_diff(got, ref)


@pytest.mark.parametrize("dim,ext,unit,bc", [(1, (5000,), 0, 0), (2, (40, 50), 3, 0), (3, (8, 9, 10), 5, 0),
                                             (3, (20, 21, 22), 2, 1)])
def test_stalled_producer_times_out_without_hanging(dim, ext, unit, bc):
    """A producer that never publishes makes its consumers' bounded waits expire: ETIMEOUT, no hang."""
    import torch
    from paper_2010_04868_gb300 import stencil as S
    w, u0 = case(dim, "star", 1, ext, seed=5)
    st = S.Stencil(dim, 0, 1, list(w), S.STENCIL_GAUSS_SEIDEL, bc).set_plan(WAVE)
    u = torch.from_numpy(u0.copy()).cuda()
    S.stencil_debug_inject_stall(st.handle, unit, 20000)
    st.run(u, 70)
    assert st.status() == S.STENCIL_ETIMEOUT
    # the handle and the context stay usable: the next run is correct again
    u.copy_(torch.from_numpy(u0))
    st.run(u, 70)
    assert st.status() == 0
    ref = oracle_run(u0, 70, dim, "star", 1, w, "gs", "periodic" if bc else "constant", 0.0, "fma")
    assert bits_equal(u.cpu().numpy(), ref)
    st.close()


PERIODIC_CASES = [(2, 1, (37, 40)), (2, 1, (130, 300)), (2, 2, (21, 33)), (3, 1, (5, 6, 7)), (3, 1, (20, 33, 40)),
                  (3, 2, (9, 10, 11))]


@pytest.mark.parametrize("dim,r,ext", PERIODIC_CASES)
def test_periodic_star_sweep_dag(dim, r, ext):
    """Periodic stars: sweeps cannot overlap; the in-sweep tile DAG in one launch matches the oracle."""
    w, u0 = case(dim, "star", r, ext, seed=dim * 10 + r + 90)
    for T in (1, 3, 8):
        for arith in ("fma", "unfused"):
            ref = oracle_run(u0, T, dim, "star", r, w, "gs", "periodic", 0.0, arith)
            got = gpu_run(u0, T, dim, "star", r, w, "gs", "periodic", 0.0, arith, plan=WAVE)
            assert bits_equal(got, ref), (T, arith, first_diff(got, ref))


def test_periodic_3d_full_size_sweep_dag_equals_plain():
    """512^3 periodic Gauss-Seidel 7-point, 6 sweeps: the one-launch DAG equals the per-diagonal plain kernel."""
    from paper_2010_04868_gb300 import inputs
    u0 = inputs.grid(inputs.SEED_BASE + 7, (512, 512, 512))
    w = inputs.normalized_weights(inputs.SEED_BASE + 208, 7)
    a = gpu_run(u0, 6, 3, "star", 1, w, "gs", "periodic", 0.0, "fma", plan=WAVE)
    b = gpu_run(u0, 6, 3, "star", 1, w, "gs", "periodic", 0.0, "fma", plan=PLAIN)
    assert bits_equal(a, b), first_diff(a, b)


def test_periodic_box_wavefront_is_rejected():
    import torch
    from paper_2010_04868_gb300 import stencil as S
    st = S.Stencil(2, 1, 1, [0.1] * 9, S.STENCIL_GAUSS_SEIDEL, S.STENCIL_BC_PERIODIC).set_plan(WAVE)
    with pytest.raises(S.StencilError) as e:
        st.run(torch.zeros(8, 8, dtype=torch.float64, device="cuda"), 3)
    assert e.value.code == S.STENCIL_EUNSUPPORTED
    st.close()


@pytest.mark.parametrize("shape,ext", [("star", (130, 77)), ("box", (70, 131))])
@pytest.mark.parametrize("tile", [(0, 0, 8), (4, 0, 8), (3, 0, 16), (0, 2, 0), (2, 5, 8), (3, 8, 16), (0, 64, 16),
                                  (4, 4, 1), (1, 0, 1), (3, 33, 1)])
def test_gs2d_wavefront_plan_parameters(shape, ext, tile):
    """Points per lane and step of the one-warp tile (8 or 16) or the decoupled tile (1, the star only),
    skewed rows per tile and CTAs per SM of the 2D wavefront change nothing in the result."""
    w, u0 = case(2, shape, 1, ext, seed=99)
    for T in (1, 33, 70):
        ref = oracle_run(u0, T, 2, shape, 1, w, "gs", "constant", 0.3, "fma")
        got = gpu_run(u0, T, 2, shape, 1, w, "gs", "constant", 0.3, "fma", plan=WAVE, tile=tile)
        assert bits_equal(got, ref), (T, first_diff(got, ref))


@pytest.mark.parametrize("ext", [(4096, 4096), (1000, 3001)])
def test_gs2d_decoupled_tile_equals_one_warp_tile(ext):
    """Full-size and ragged 2D 5-point grids, 70 sweeps (two full sweep blocks and a partial one): the
    decoupled tile (chain, producer and scheduler warps) and the one-warp tile agree bit for bit."""
    from paper_2010_04868_gb300 import inputs
    u0 = inputs.grid(inputs.SEED_BASE + 31, ext)
    w = inputs.normalized_weights(inputs.SEED_BASE + 131, 5)
    for arith in ("fma", "unfused"):
        a = gpu_run(u0, 70, 2, "star", 1, w, "gs", "constant", 0.2, arith, plan=WAVE, tile=(0, 0, 1))
        b = gpu_run(u0, 70, 2, "star", 1, w, "gs", "constant", 0.2, arith, plan=WAVE)
        assert bits_equal(a, b), (arith, first_diff(a, b))


@pytest.mark.parametrize("dim,r,ext,tile", [(3, 1, (13, 11, 17), (4, 8, 16)), (3, 1, (20, 9, 12), (1, 32, 8)),
                                            (3, 2, (11, 12, 13), (2, 16, 5)), (2, 1, (70, 45), (0, 32, 32)),
                                            (2, 2, (33, 40), (0, 32, 7))])
def test_periodic_sweep_dag_tile_shapes(dim, r, ext, tile):
    """The in-sweep DAG with the tile shape a plan fixes (lines per tile along axes 0 and 1, hyperplane steps)."""
    w, u0 = case(dim, "star", r, ext, seed=dim * 31 + r)
    ref = oracle_run(u0, 5, dim, "star", r, w, "gs", "periodic", 0.0, "fma")
    got = gpu_run(u0, 5, dim, "star", r, w, "gs", "periodic", 0.0, "fma", plan=WAVE, tile=tile)
    assert bits_equal(got, ref), first_diff(got, ref)


ROWS = (0, 0, 2)   # wavefront plan: rows as lanes


@pytest.mark.parametrize("shape,ext", [("star", (1, 4)), ("star", (1, 68)), ("star", (70, 4)), ("star", (32, 64)),
                                       ("star", (33, 68)), ("star", (130, 76)), ("star", (31, 200)),
                                       ("box", (1, 4)), ("box", (2, 8)), ("box", (64, 32)), ("box", (70, 132)),
                                       ("box", (97, 36)), ("star", (33, 65)), ("box", (70, 131)), ("star", (5, 2))])
@pytest.mark.parametrize("c", [0.0, 0.3])
def test_gs2d_rows_equals_oracle(shape, ext, c):
    """Rows as lanes (tile[2] = 2): ragged bands and rows shorter than the lanes' skew, both rounding modes;
    rows that are not whole groups of four columns take the one-warp tiles instead."""
    w, u0 = case(2, shape, 1, ext, seed=ext[0] + 3 * ext[1])
    for T in (1, 2, 5, 33):
        for arith in ("fma", "unfused"):
            ref = oracle_run(u0, T, 2, shape, 1, w, "gs", "constant", c, arith)
            got = gpu_run(u0, T, 2, shape, 1, w, "gs", "constant", c, arith, plan=WAVE, tile=ROWS)
            assert bits_equal(got, ref), (T, arith, first_diff(got, ref))


@pytest.mark.parametrize("shape", ["star", "box"])
@pytest.mark.parametrize("tile", [(1, 0, 2), (2, 0, 2), (6, 0, 2), (4, 64, 2), (3, 128, 2), (1, 128, 2), (3, 16, 2), (3, 0, 2)])
def test_gs2d_rows_plan_parameters(shape, tile):
    """The CTAs per SM (tile[0]) and the steps per chunk (tile[1]: 16, 64 or 128; 8 by default) a plan asks for change
    nothing in the result."""
    w, u0 = case(2, shape, 1, (300, 256), seed=5)
    ref = oracle_run(u0, 40, 2, shape, 1, w, "gs", "constant", 0.1, "fma")
    got = gpu_run(u0, 40, 2, shape, 1, w, "gs", "constant", 0.1, "fma", plan=WAVE, tile=tile)
    assert bits_equal(got, ref), first_diff(got, ref)


@pytest.mark.parametrize("shape", ["star", "box"])
def test_gs2d_rows_full_size_equals_oracle(shape):
    """The 4096^2 Gauss-Seidel workload's grid with rows as lanes, T cut to 24 for the serial oracle."""
    from paper_2010_04868_gb300 import inputs
    u0 = inputs.grid(inputs.SEED_BASE + 3, (4096, 4096))
    w = inputs.normalized_weights(inputs.SEED_BASE + 105, 5 if shape == "star" else 9)
    ref = oracle_run(u0, 24, 2, shape, 1, w, "gs", "constant", 0.0, "fma")
    got = gpu_run(u0, 24, 2, shape, 1, w, "gs", "constant", 0.0, "fma", plan=WAVE, tile=ROWS)
    assert bits_equal(got, ref), first_diff(got, ref)


def test_gs2d_rows_full_size_full_T_equals_plain():
    """Full 4096^2 x 200 sweeps: rows as lanes and the plain sweep kernel agree bit for bit."""
    from paper_2010_04868_gb300 import inputs
    u0 = inputs.grid(inputs.SEED_BASE + 3, (4096, 4096))
    w = inputs.normalized_weights(inputs.SEED_BASE + 105, 5)
    a = gpu_run(u0, 200, 2, "star", 1, w, "gs", "constant", 0.0, "fma", plan=WAVE, tile=ROWS)
    b = gpu_run(u0, 200, 2, "star", 1, w, "gs", "constant", 0.0, "fma", plan=PLAIN)
    assert bits_equal(a, b), first_diff(a, b)


def test_gs2d_rows_stalled_task_times_out_without_hanging():
    """A task that never publishes its progress: the tasks waiting on it give up (bounded), the run
    reports STENCIL_ETIMEOUT, and the next run on the same handle is correct."""
    import torch
    from paper_2010_04868_gb300 import stencil as S
    w, u0 = case(2, "star", 1, (100, 92), seed=8)
    st = S.Stencil(2, 0, 1, list(w), S.STENCIL_GAUSS_SEIDEL, S.STENCIL_BC_CONSTANT, 0.0).set_plan(WAVE, 0, ROWS)
    u = torch.from_numpy(u0.copy()).cuda()
    S.stencil_debug_inject_stall(st.handle, 3, 20000)
    st.run(u, 6)
    assert st.status() == S.STENCIL_ETIMEOUT
    u.copy_(torch.from_numpy(u0))
    st.run(u, 6)
    assert st.status() == S.STENCIL_OK
    ref = oracle_run(u0, 6, 2, "star", 1, w, "gs", "constant", 0.0, "fma")
    assert bits_equal(u.cpu().numpy(), ref)
    st.close()


def test_gs2d_rows_many_sweeps_split_over_launches():
    """More sweeps than one launch's progress words hold (2^18 tasks: 131072 sweeps of a 2-band grid):
    the rows pipeline runs them in two launches and agrees with the one-warp tiles bit for bit."""
    w, u0 = case(2, "star", 1, (64, 64), seed=21)
    T = (1 << 17) + 5
    a = gpu_run(u0, T, 2, "star", 1, w, "gs", "constant", 0.1, "fma", plan=WAVE, tile=ROWS)
    b = gpu_run(u0, T, 2, "star", 1, w, "gs", "constant", 0.1, "fma", plan=WAVE, tile=(0, 0, 16))
    assert bits_equal(a, b), first_diff(a, b)


@pytest.mark.parametrize("ext", [(1, 4), (2, 8), (3, 12), (31, 64), (33, 68), (64, 36), (97, 132), (130, 76)])
@pytest.mark.parametrize("c", [0.0, 0.3])
def test_gs2d_rows_radius2_star_equals_oracle(ext, c):
    """Rows as lanes for the 9-point star of radius 2 (lanes 0/1 and 30/31 reach two rows beyond the
    band): ragged bands, both rounding modes, bit for bit."""
    w, u0 = case(2, "star", 2, ext, seed=ext[0] + 5 * ext[1])
    for T in (1, 2, 5, 33):
        for arith in ("fma", "unfused"):
            ref = oracle_run(u0, T, 2, "star", 2, w, "gs", "constant", c, arith)
            got = gpu_run(u0, T, 2, "star", 2, w, "gs", "constant", c, arith, plan=WAVE, tile=ROWS)
            assert bits_equal(got, ref), (T, arith, first_diff(got, ref))


def test_gs2d_rows_radius2_full_size_equals_oracle():
    """The 4096^2 radius-2 Gauss-Seidel workload's grid with rows as lanes (its default plan), T cut to 12."""
    from paper_2010_04868_gb300 import inputs
    u0 = inputs.grid(inputs.SEED_BASE + 3, (4096, 4096))
    w = inputs.normalized_weights(inputs.SEED_BASE + 319, 9)
    ref = oracle_run(u0, 12, 2, "star", 2, w, "gs", "constant", 0.0, "fma")
    got = gpu_run(u0, 12, 2, "star", 2, w, "gs", "constant", 0.0, "fma", plan=WAVE)
    assert bits_equal(got, ref), first_diff(got, ref)
