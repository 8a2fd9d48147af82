"""CPU restatement of the cell walk in the temporally blocked Jacobi kernels.

Each step of a blocked pass (csrc/k_blocked.cu, and the pass units of csrc/k_batch.cu) updates the
cells of the staged region that are still valid after s steps: a box [lo, hi) that shrinks by r per
step on every used axis. Thread t of nthr takes the cells t, t + nthr, t + 2 nthr, ... of that box
in row-major order. In 2D and 3D the kernels do not divide per cell: each thread decodes its first
cell once, splits the stride nthr into digits (dq0, dq1, dr) of the box's mixed radix (w1, w2), and
adds them with carries. In 1D the loop runs over the cells themselves.

These tests restate that walk and check, on the geometries the hosts build (the tile plus a halo of
T_b r per side; in k_blocked.cu the inner axis padded by one cell when its start is rounded down to
an even index, and the 1D region rounded up to a multiple of 256), that every thread visits exactly
the cells of the row-major decode of its indices, so the box is covered once with no cell twice, and
that no coordinate leaves [lo, hi).
"""
import itertools

import pytest


def walk(lo, hi, tid, nthr):
    """Cells visited by thread tid: the 2D/3D carry walk of the kernels' step loop."""
    lo0, lo1, lo2 = lo
    hi0, hi1, hi2 = hi
    w1, w2 = hi1 - lo1, hi2 - lo2
    cnt = (hi0 - lo0) * w1 * w2
    dr, dq = nthr % w2, nthr // w2
    dq1, dq0 = dq % w1, dq // w1
    s2 = lo2 + tid % w2
    s1 = lo1 + (tid // w2) % w1
    s0 = lo0 + tid // (w2 * w1)
    out = []
    idx = tid
    while idx < cnt:
        out.append((s0, s1, s2))
        s2 += dr
        s1 += dq1
        s0 += dq0
        if s2 >= hi2:
            s2 -= w2
            s1 += 1
        if s1 >= hi1:
            s1 -= w1
            s0 += 1
        idx += nthr
    return out


def walk_1d(lo2, hi2, tid, nthr):
    """Cells visited by thread tid in 1D: the loop over the cells themselves."""
    return [(0, 0, s2) for s2 in range(lo2 + tid, hi2, nthr)]


def decode(lo, hi, idx):
    """Row-major cell idx of the box [lo, hi): the division decode the walk replaces."""
    w1, w2 = hi[1] - lo[1], hi[2] - lo[2]
    return (lo[0] + idx // (w1 * w2), lo[1] + (idx // w2) % w1, lo[2] + idx % w2)


def step_boxes(dim, r, tile, tb, pad2, e2_extra):
    """Per-step valid boxes of one staged region, as the kernels compute them."""
    h = [tb * r if dim >= 3 else 0, tb * r if dim >= 2 else 0, tb * r]
    B = [tile[0] if dim >= 3 else 1, tile[1] if dim >= 2 else 1, tile[2]]
    E = [B[0] + 2 * h[0], B[1] + 2 * h[1], B[2] + 2 * h[2] + e2_extra]
    if dim == 1 and e2_extra:
        E[2] = (E[2] + 255) & ~255
    for s in range(1, tb + 1):
        lo = (s * r if dim >= 3 else 0, s * r if dim >= 2 else 0, pad2 + s * r)
        hi = (E[0] - s * r if dim >= 3 else 1, E[1] - s * r if dim >= 2 else 1, pad2 + B[2] + 2 * h[2] - s * r)
        yield lo, hi, E


def check_box(dim, lo, hi, E, nthr):
    cnt = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
    assert cnt > 0
    seen = set()
    for t in range(nthr):
        cells = walk_1d(lo[2], hi[2], t, nthr) if dim == 1 else walk(lo, hi, t, nthr)
        want = [decode(lo, hi, i) for i in range(t, cnt, nthr)]
        assert cells == want, (dim, lo, hi, t)
        for c in cells:
            assert all(lo[a] <= c[a] < hi[a] for a in range(3)), (c, lo, hi)
            assert all(0 <= c[a] < E[a] for a in range(3)), (c, E)
            assert c not in seen
            seen.add(c)
    assert len(seen) == cnt


BLOCKED_CASES = [
    # dim, r, tile, tb
    (1, 1, (0, 0, 256), 64),
    (1, 1, (0, 0, 108), 32),
    (1, 2, (0, 0, 37), 5),
    (2, 1, (0, 32, 128), 4),
    (2, 1, (0, 7, 300), 3),
    (2, 2, (0, 16, 5), 2),
    (2, 1, (0, 1, 1), 1),
    (3, 1, (8, 8, 16), 2),
    (3, 2, (3, 5, 7), 2),
    (3, 1, (16, 4, 64), 1),
]


@pytest.mark.parametrize("dim,r,tile,tb", BLOCKED_CASES)
@pytest.mark.parametrize("pad2", [0, 1])
def test_blocked_kernel_walk_covers_each_step_once(dim, r, tile, tb, pad2):
    """k_jacobi_blocked: 256 threads, the inner axis padded for the rounded TMA start."""
    for lo, hi, E in step_boxes(dim, r, tile, tb, pad2, e2_extra=2):
        check_box(dim, lo, hi, E, 256)


@pytest.mark.parametrize("dim,r,tile,tb", BLOCKED_CASES)
def test_batch_pass_unit_walk_covers_each_step_once(dim, r, tile, tb):
    """The batched kernel's pass units: 256 threads, no padding of the inner axis."""
    for lo, hi, E in step_boxes(dim, r, tile, tb, 0, e2_extra=0):
        check_box(dim, lo, hi, E, 256)


@pytest.mark.parametrize("nthr", [32, 96, 256, 1024])
def test_walk_any_stride(nthr):
    """The carry walk equals the decode for strides below, between and above the box's digits."""
    for w0, w1, w2 in itertools.product((1, 2, 5), (1, 3, 17, 40), (1, 2, 31, 33, 257)):
        lo = (2, 1, 3)
        hi = (lo[0] + w0, lo[1] + w1, lo[2] + w2)
        cnt = w0 * w1 * w2
        for t in range(min(nthr, cnt)):
            assert walk(lo, hi, t, nthr) == [decode(lo, hi, i) for i in range(t, cnt, nthr)], (nthr, w0, w1, w2, t)


def test_planted_carry_mistake_is_caught():
    """A walk that forgets the carry from the inner digit visits the wrong cells: the comparison sees it."""
    lo, hi, nthr = (0, 0, 0), (1, 40, 20), 256      # 800 cells: every thread takes several

    def bad_walk(t):
        w1, w2 = hi[1] - lo[1], hi[2] - lo[2]
        cnt = w1 * w2
        dr, dq = nthr % w2, nthr // w2
        s2, s1 = t % w2, (t // w2) % w1
        out, idx = [], t
        while idx < cnt:
            out.append((0, s1, s2))
            s2 += dr
            s1 += dq
            if s2 >= hi[2]:
                s2 -= w2          # the carry into s1 is missing
            idx += nthr
        return out

    cnt = 40 * 20
    assert any(bad_walk(t) != [decode(lo, hi, i) for i in range(t, cnt, nthr)] for t in range(nthr))
