"""LCS (Section 3.4) on the GPU: both wavefront kernels against the oracle's last row, exactly, through the C ABI."""
import ctypes

import numpy as np
import pytest

import oracle.integer as OI
from paper_2010_04868_gb300 import inputs

pytestmark = pytest.mark.gpu

DP, BITS, AUTO = 1, 2, 0


def _gpu(A, B, kernel, workspace=False):
    import torch
    from paper_2010_04868_gb300 import lcs
    a = torch.from_numpy(np.ascontiguousarray(A, np.uint8)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(B, np.uint8)).cuda()
    ws = None
    if workspace:
        ws = torch.empty(lcs.lcs_workspace_bytes(len(A), len(B), kernel), dtype=torch.uint8, device="cuda")
    row = lcs.run(a, b, kernel, workspace=ws)
    if ws is not None:
        assert lcs.lcs_status(ctypes.c_void_p(ws.data_ptr())) == 0
    torch.cuda.synchronize()
    return row.cpu().numpy()


SIZES = [(1, 1), (1, 100), (100, 1), (31, 33), (32, 64), (33, 65), (255, 256), (257, 129), (300, 2000), (1000, 70),
         (2049, 4100)]


@pytest.mark.parametrize("na,nb", SIZES)
@pytest.mark.parametrize("kernel", [DP, BITS])
@pytest.mark.parametrize("sigma", [2, 4, 256])
def test_lcs_row(na, nb, kernel, sigma):
    A = inputs.sequence(2000 + na, na, sigma)
    B = inputs.sequence(3000 + nb, nb, sigma)
    ref = OI.lcs(A, B)
    got = _gpu(A, B, kernel)
    assert np.array_equal(got, ref), (np.argwhere(got != ref)[:5], got[-1], ref[-1])


@pytest.mark.parametrize("kernel", [DP, BITS, AUTO])
def test_lcs_edge_cases(kernel):
    for A, B in ((b"", b"abc"), (b"abc", b""), (b"", b""), (b"ABCBDAB", b"BDCABA"), (b"a" * 70, b"a" * 130),
                 (b"ab" * 40, b"ba" * 33)):
        a = np.frombuffer(A, np.uint8)
        b = np.frombuffer(B, np.uint8)
        assert np.array_equal(_gpu(a, b, kernel), OI.lcs(a, b)), (A[:8], B[:8])


@pytest.mark.parametrize("kernel", [DP, BITS])
def test_lcs_with_workspace_and_status(kernel):
    A = inputs.sequence(4001, 700, 4)
    B = inputs.sequence(4002, 900, 4)
    assert np.array_equal(_gpu(A, B, kernel, workspace=True), OI.lcs(A, B))


def test_lcs_argument_errors():
    import torch
    from paper_2010_04868_gb300 import stencil as S
    lib = S.load()
    a = torch.zeros(10, dtype=torch.uint8, device="cuda")
    row = torch.zeros(11, dtype=torch.int32, device="cuda")
    pa, pr = ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(row.data_ptr())
    assert lib.lcs_run(pa, -1, pa, 10, pr, 0, None, None) == S.STENCIL_EINVAL
    assert lib.lcs_run(pa, 10, pa, 10, None, 0, None, None) == S.STENCIL_EINVAL
    assert lib.lcs_run(pa, 10, pa, 10, pr, 7, None, None) == S.STENCIL_EINVAL
    assert lib.lcs_run(None, 10, pa, 10, pr, 0, None, None) == S.STENCIL_EINVAL
    assert lib.lcs_run(pa, 10, pa, 10, pr, 0, ctypes.c_void_p(row.data_ptr() + 4), None) == S.STENCIL_EINVAL
    assert lib.lcs_run(pa, (1 << 30) + 1, pa, 10, pr, 0, None, None) == S.STENCIL_EINVAL


@pytest.mark.parametrize("kernel", [DP, BITS])
def test_lcs_large(kernel):
    """20000 x 30000 over 4 symbols: thousands of strips in flight, rows recycled through the ring."""
    A = inputs.sequence(inputs.SEED_BASE + 600, 20000, 4)
    B = inputs.sequence(inputs.SEED_BASE + 601, 30000, 4)
    assert np.array_equal(_gpu(A, B, kernel), OI.lcs(A, B))
