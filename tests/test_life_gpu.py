"""Game of Life (Section 3.4) on the GPU: the bit-packed kernels against the oracle, bit for bit, through the C ABI."""
import ctypes

import numpy as np
import pytest

import oracle.integer as OI
from paper_2010_04868_gb300 import inputs

pytestmark = pytest.mark.gpu

RULES = {"b2s23": OI.B2S23, "b3s23": OI.B3S23, "other": (0b000001010, 0b000110100), "all": (0x1FF, 0x1FF)}


def _gpu(c0, T, bc, rule, tb):
    import torch
    from paper_2010_04868_gb300 import life
    t = torch.from_numpy(np.ascontiguousarray(c0)).cuda()
    life.run(t, T, boundary=bc, rule=rule, tb=tb)
    torch.cuda.synchronize()
    return t.cpu().numpy()


SIZES = [(1, 1), (1, 70), (70, 1), (3, 3), (5, 64), (7, 65), (33, 127), (130, 200), (64, 128), (150, 4100),
         (70, 3968), (66, 4032)]


@pytest.mark.parametrize("ext", SIZES)
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("tb", [1, 0, 5])
def test_life_b2s23(ext, bc, tb):
    if bc == 1 and min(ext) < 3:
        pytest.skip("periodic grids need extents >= 3")
    c0 = inputs.cells(1000 + ext[0] + 7 * ext[1], ext, 0.4)
    for T in (1, 2, 17, 40):
        ref = OI.life(c0, T, bc=bc, rule=OI.B2S23)
        got = _gpu(c0, T, bc, OI.B2S23, tb)
        assert np.array_equal(got, ref), (T, np.argwhere(got != ref)[:5])


@pytest.mark.parametrize("rule", sorted(RULES))
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("tb", [1, 16, 64])
def test_life_rules(rule, bc, tb):
    ext = (97, 320) if bc == 1 else (97, 300)   # periodic: a whole number of words, so the blocked kernel runs
    c0 = inputs.cells(1100 + len(rule), ext, 0.35)
    for T in (3, 64, 70):
        ref = OI.life(c0, T, bc=bc, rule=RULES[rule])
        got = _gpu(c0, T, bc, RULES[rule], tb)
        assert np.array_equal(got, ref), (rule, T)


def test_life_periodic_ragged_width_falls_back_to_one_step_kernel():
    c0 = inputs.cells(1201, (40, 100), 0.4)     # 100 cells: not a whole number of 64-cell words
    ref = OI.life(c0, 33, bc=1)
    assert np.array_equal(_gpu(c0, 33, 1, OI.B2S23, 16), ref)


def test_life_glider_circles_a_torus():
    g = np.zeros((64, 64), np.uint8)
    g[0:3, 0:3] = [[0, 1, 0], [0, 0, 1], [1, 1, 1]]
    assert np.array_equal(_gpu(g, 4 * 64, 1, OI.B3S23, 0), g)


def test_life_nonbinary_bytes_read_as_live():
    c0 = inputs.cells(1211, (20, 30), 0.5) * np.uint8(7)
    got = _gpu(c0, 3, 0, OI.B2S23, 0)
    assert np.array_equal(got, OI.life((c0 != 0).astype(np.uint8), 3))
    assert set(np.unique(got)) <= {0, 1}


def test_life_workspace_and_errors():
    import torch
    from paper_2010_04868_gb300 import life
    from paper_2010_04868_gb300 import stencil as S
    c0 = inputs.cells(1221, (50, 130), 0.4)
    t = torch.from_numpy(c0).cuda()
    nbytes = life.life_workspace_bytes((50, 130))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    life.run(t, 9, workspace=ws)
    assert np.array_equal(t.cpu().numpy(), OI.life(c0, 9))
    before = t.clone()
    life.run(t, 0)
    assert torch.equal(t, before)
    lib = S.load()
    e = (ctypes.c_int64 * 2)(50, 130)
    p = ctypes.c_void_p(t.data_ptr())
    assert lib.life_run(p, e, 0, 0x200, 0, 1, 0, None, None) == S.STENCIL_EINVAL
    assert lib.life_run(p, e, 0, 4, 12, -1, 0, None, None) == S.STENCIL_EINVAL
    assert lib.life_run(p, e, 2, 4, 12, 1, 0, None, None) == S.STENCIL_EINVAL
    e2 = (ctypes.c_int64 * 2)(2, 130)
    assert lib.life_run(p, e2, 1, 4, 12, 1, 0, None, None) == S.STENCIL_EINVAL
    assert lib.life_run(p, e, 0, 4, 12, 1, 0, ctypes.c_void_p(ws.data_ptr() + 8), None) == S.STENCIL_EINVAL
    assert lib.life_run(None, e, 0, 4, 12, 1, 0, None, None) == S.STENCIL_EINVAL


def test_life_full_size():
    """The 8000^2 B2S23 workload in its launch configuration (default steps per launch), T cut to 40."""
    c0 = inputs.cells(inputs.SEED_BASE + 500, (8000, 8000), 0.5)
    ref = OI.life(c0, 40)
    got = _gpu(c0, 40, 0, OI.B2S23, 0)
    assert np.array_equal(got, ref)
