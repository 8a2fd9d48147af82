"""The autotuned default plan gives the oracle's result, and the tuning cache round-trips through its file."""
import json
import os
import subprocess
import sys

import pytest

from helpers import bits_equal, case, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("dim,shape,ext,T", [(1, "star", (65536,), 256), (2, "star", (300, 200), 30),
                                             (3, "box", (40, 30, 50), 6)])
def test_auto_plan_matches_oracle(dim, shape, ext, T):
    w, u0 = case(dim, shape, 1, ext, seed=81)
    ref = oracle_run(u0, T, dim, shape, 1, w, "jacobi", "constant", 0.0, "fma")
    got = gpu_run(u0, T, dim, shape, 1, w, "jacobi", "constant", 0.0, "fma", plan=None)
    assert bits_equal(got, ref)


def test_tune_cache_file(tmp_path):
    cache = tmp_path / "tune.jsonl"
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import torch\n"
        "from paper_2010_04868_gb300 import stencil as S\n"
        "st = S.Stencil(1, 0, 1, [0.25, 0.5, 0.25])\n"
        "u = torch.rand(65536, dtype=torch.float64, device='cuda')\n"
        "st.run(u, 256); torch.cuda.synchronize(); print('ok')\n" % ROOT)
    env = dict(os.environ, STENCIL_TUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = [json.loads(x) for x in cache.read_text().splitlines()]
    assert len(lines) == 1 and lines[0]["kernel"] in (1, 2, 4)
    # a second process reads the entry instead of tuning again
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert len(cache.read_text().splitlines()) == 1


def test_get_plan_reports_fixed_and_tuned_plans():
    import torch
    from paper_2010_04868_gb300 import stencil as S
    st = S.Stencil(2, 1, 1, [1.0 / 9] * 9)
    u = torch.rand(200, 300, dtype=torch.float64, device="cuda")
    st.set_plan(S.STENCIL_KERNEL_DIAMOND, 6, (0, 40, 50))
    assert st.plan(u, 30) == (S.STENCIL_KERNEL_DIAMOND, 6, (0, 40, 50))
    st.set_plan(S.STENCIL_KERNEL_AUTO)
    k, tb, tile = st.plan(u, 30)
    assert k in (S.STENCIL_KERNEL_PLAIN, S.STENCIL_KERNEL_BLOCKED, S.STENCIL_KERNEL_DIAMOND,
                 S.STENCIL_KERNEL_STREAM) and tb >= 1
    assert st.plan(u, 30) == (k, tb, tile)          # cached: the same answer without tuning again
    gs = S.Stencil(2, 0, 1, [0.2] * 5, S.STENCIL_GAUSS_SEIDEL)
    assert gs.plan(u, 10)[0] == S.STENCIL_KERNEL_WAVEFRONT
    gp = S.Stencil(2, 0, 1, [0.2] * 5, S.STENCIL_GAUSS_SEIDEL, S.STENCIL_BC_PERIODIC)
    assert gp.plan(u, 10)[0] in (S.STENCIL_KERNEL_WAVEFRONT, S.STENCIL_KERNEL_PLAIN)
    for x in (st, gs, gp):
        x.close()


# the wavefront Gauss-Seidel parameter sets the tuner times (the first is the default)
GS_2D_STAR1 = [(0, 0, 0), (3, 16, 16), (4, 16, 16), (3, 8, 16), (2, 32, 8), (3, 32, 1)]


@pytest.mark.parametrize("dim,shape,ext,T", [(2, "star", (700, 520), 70), (2, "box", (300, 410), 40),
                                             (3, "star", (40, 50, 60), 33)])
def test_auto_gauss_seidel_plan_is_timed_and_matches_oracle(dim, shape, ext, T):
    """An automatic Gauss-Seidel plan is one of the timed wavefront parameter sets, and gives the oracle's
    result bit for bit."""
    import torch
    from paper_2010_04868_gb300 import stencil as S
    w, u0 = case(dim, shape, 1, ext, seed=91)
    st = S.Stencil(dim, 0 if shape == "star" else 1, 1, list(w), S.STENCIL_GAUSS_SEIDEL)
    u = torch.from_numpy(u0.copy()).cuda()
    k, tb, tile = st.plan(u, T)
    assert k == S.STENCIL_KERNEL_WAVEFRONT
    if dim == 2 and shape == "star":
        assert tuple(tile) in GS_2D_STAR1
    elif dim == 3:
        assert tile[0] in (0, 3, 4)
    st.run(u, T)
    assert st.status() == 0
    ref = oracle_run(u0, T, dim, shape, 1, w, "gs", "constant", 0.0, "fma")
    assert bits_equal(u.cpu().numpy(), ref)
    st.close()
