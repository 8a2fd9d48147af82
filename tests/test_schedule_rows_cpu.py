"""CPU restatement of the rows-as-lanes 2D Gauss-Seidel pipeline (k_gs2d_rows in csrc/k_wavefront.cu).

A task (s, b) is sweep s over band b (32 rows, one per lane); at step t lane k updates the group of four
columns G = t - SK k (SK = 1 for the stars of radius 1 ("star") and 2 ("star2"), 2 for the box). Each chunk of ch steps (8 by default; 16, 64 or
128 when a plan asks) first waits for the progress of (s, b-1), (s-1, b) and (s-1, b+1), then runs,
then publishes. Every load a chunk issues (a lane's own row four groups ahead, lane 0's row above and
lane 31's row below three or four groups ahead, and the first chunk's ring fill) and every store is
placed in the chunk that issues it. The checks, on small ragged grids:
  * every wait names a task with an earlier ticket (tickets in the order (s + b, s)), so the
    persistent kernel cannot deadlock;
  * any two chunks the waits (and program order) leave unordered touch disjoint points: neither
    writes a point the other reads or writes; as the compiler may move a chunk's loads up to its
    wait and its stores down to its publication, this covers every timing the kernel can have;
  * running the chunks in random orders that respect the waits, with the lanes' register rings and
    shuffles emulated step by step, gives the oracle's result bit for bit (unfused rounding, which
    Python floats reproduce exactly).
"""
import numpy as np
import pytest

from helpers import case, oracle_run
from paper_2010_04868_gb300 import inputs


def params(shape):
    """(SK, QX0, LX): lane skew in groups, first group of the x-row rings and the group they load."""
    return {"star": (1, 0, 4), "box": (2, -1, 3), "star2": (1, -1, 3)}[shape]


def radius(shape):
    return 2 if shape == "star2" else 1


def geometry(n0, n1, T, ch, shape):
    sk = params(shape)[0]
    nb = -(-n0 // 32)
    ng = n1 // 4
    steps = -(-(ng + 31 * sk) // ch) * ch
    order = [(s, e - s) for e in range(T + nb - 1) for s in range(max(0, e - nb + 1), min(T - 1, e) + 1)]
    return nb, ng, steps, order


def chunk_waits(s, b, t0, nb, ng, ch, shape):
    """(task, progress needed) pairs a chunk starting at step t0 waits for (the kernel's nA, nO, nB)."""
    sk, _, lx = params(shape)
    smax = ng + 31 * sk
    out = []
    nA, nO, nB = t0 + ch + lx + 31 * sk, t0 + ch + 4, t0 + ch - 31 * sk + lx + radius(shape) - 1
    if b > 0:
        out.append(((s, b - 1), min(nA, smax)))
    if s > 0:
        out.append(((s - 1, b), min(nO, smax)))
    if s > 0 and b + 1 < nb and nB > 0:
        out.append(((s - 1, b + 1), min(nB, smax)))
    return out


def chunk_access(s, b, c, n0, ng, ch, shape):
    """Points a chunk reads and writes."""
    sk, qx0, lx = params(shape)
    rd, wr = set(), set()

    def add(row, grp, into):
        if 0 <= row < n0 and 0 <= grp < ng:
            for x in range(4):
                into.add((row, 4 * grp + x))
    t0 = c * ch
    if c == 0:
        for k in range(32):
            for q in range(4):
                add(32 * b + k, -sk * k + q, rd)
        for q in range(qx0, qx0 + 4):
            for d in range(radius(shape)):
                add(32 * b - 1 - d, q, rd)
                add(32 * b + 32 + d, -31 * sk + q, rd)
    for t in range(t0, t0 + ch):
        for k in range(32):
            g = t - sk * k
            add(32 * b + k, g, wr)
            add(32 * b + k, g + 4, rd)
        for d in range(radius(shape)):
            add(32 * b - 1 - d, t + lx, rd)
            add(32 * b + 32 + d, t - 31 * sk + lx, rd)
    return rd, wr


CASES = [(40, 36, 3), (64, 52, 3), (33, 68, 3), (5, 8, 4), (70, 12, 3), (70, 152, 3), (96, 40, 2), (1, 4, 2)]


@pytest.mark.parametrize("shape", ["star", "box", "star2"])
@pytest.mark.parametrize("ch", [8, 16, 32, 64])
@pytest.mark.parametrize("n0,n1,T", CASES)
def test_waits_point_back_and_unordered_chunks_do_not_conflict(n0, n1, T, ch, shape):
    nb, ng, steps, order = geometry(n0, n1, T, ch, shape)
    ticket = {x: q for q, x in enumerate(order)}
    nch = steps // ch
    inst = [(x, c) for x in order for c in range(nch)]
    idx = {v: q for q, v in enumerate(inst)}
    pred = [0] * len(inst)
    acc = []
    for q, ((s, b), c) in enumerate(inst):
        p = 0
        if c > 0:
            p |= pred[idx[((s, b), c - 1)]] | (1 << idx[((s, b), c - 1)])
        for (y, need) in chunk_waits(s, b, c * ch, nb, ng, ch, shape):
            assert ticket[y] < ticket[(s, b)], "a wait names a later ticket"
            cy = -(-need // ch) - 1          # the chunk whose publication first reaches need
            assert 0 <= cy < nch
            p |= pred[idx[(y, cy)]] | (1 << idx[(y, cy)])
        pred[q] = p
        acc.append(chunk_access(s, b, c, n0, ng, ch, shape))
    for a in range(len(inst)):
        ra, wa = acc[a]
        for bq in range(a + 1, len(inst)):
            if (pred[bq] >> a) & 1 or (pred[a] >> bq) & 1:
                continue
            rb, wb = acc[bq]
            assert not (wa & (rb | wb)), (inst[a], inst[bq])
            assert not (wb & ra), (inst[a], inst[bq])


def run_chunk(state, u, s, b, c, w_desc, cval, shape, n0, ng, ch):
    """One chunk of task (s, b), the lanes' registers emulated as the kernel holds them: RO[(m + q) & 3]
    own-row old group G + q, RX[(m + q) & 3] the x row's group G + q (RY the second row beyond the band,
    radius 2), O[m & 3] the outputs of step m."""
    sk, qx0, lx = params(shape)
    RO, RX, RY, O = state
    xrow = [32 * b - 1 if k == 0 else 32 * b + 32 for k in range(32)]
    yrow = [32 * b - 2 if k == 0 else 32 * b + 33 for k in range(32)]

    def ld(row, grp):
        if 0 <= row < n0 and 0 <= grp < ng:
            return [u[row, 4 * grp + x] for x in range(4)]
        return [cval] * 4
    if c == 0:
        for k in range(32):
            for q in range(4):
                RO[k][q] = ld(32 * b + k, -sk * k + q)
            for q in range(qx0, qx0 + 4):
                RX[k][q & 3] = ld(xrow[k], -sk * k + q) if k in (0, 31) else [cval] * 4
                RY[k][q & 3] = ld(yrow[k], -sk * k + q) if k in (0, 31) and shape == "star2" else [cval] * 4
            O[k] = [[cval] * 4 for _ in range(4)]
    for tg in range(c * ch, c * ch + ch, 4):
        for m in range(4):
            outs = []
            for k in range(32):
                def dn(slot):      # __shfl_down_sync(RO[slot], 1); lane 31 keeps its own value
                    return RO[k + 1][slot] if k < 31 else RO[k][slot]

                def up(slot):      # __shfl_up_sync(O[slot], 1); lane 0 keeps its own value
                    return O[k - 1][slot] if k > 0 else O[k][slot]
                cen = RO[k][m & 3]
                rgt = cen[1:] + [RO[k][(m + 1) & 3][0]]
                left = O[k][(m + 3) & 3][3]
                out = []
                if shape == "star2":
                    b1 = RX[k][m & 3] if k == 31 else dn((m + 1) & 3)
                    if k == 31:
                        b2 = RY[k][m & 3]
                    elif k == 30:
                        b2 = RX[31][(m + 1) & 3]          # lane 31's x row at its q = +1
                    else:
                        b2 = RO[k + 2][(m + 2) & 3]
                    a1 = RX[k][m & 3] if k == 0 else up((m + 3) & 3)
                    if k == 0:
                        a2 = RY[k][m & 3]
                    elif k == 1:
                        a2 = RX[0][(m + 3) & 3]           # lane 0's x row at its q = -1
                    else:
                        a2 = O[k - 2][(m + 2) & 3]
                    l2 = O[k][(m + 3) & 3][2]
                    r2 = cen[2:] + RO[k][(m + 1) & 3][:2]
                    for x in range(4):
                        vals = [b2[x], b1[x], r2[x], rgt[x], cen[x], left, l2, a1[x], a2[x]]
                        a = w_desc[0] * vals[0]
                        for wq, v in zip(w_desc[1:], vals[1:]):
                            a = a + wq * v
                        out.append(a)
                        l2 = left
                        left = a
                elif shape == "star":
                    bel = RX[k][m & 3] if k == 31 else dn((m + 1) & 3)
                    abv = RX[k][m & 3] if k == 0 else up((m + 3) & 3)
                    for x in range(4):
                        vals = [bel[x], rgt[x], cen[x], left, abv[x]]
                        a = w_desc[0] * vals[0]
                        for wq, v in zip(w_desc[1:], vals[1:]):
                            a = a + wq * v
                        out.append(a)
                        left = a
                else:
                    if k == 31:
                        bv = [RX[k][(m + 3) & 3][3]] + RX[k][m & 3] + [RX[k][(m + 1) & 3][0]]
                    else:
                        bv = [dn((m + 1) & 3)[3]] + dn((m + 2) & 3) + [dn((m + 3) & 3)[0]]
                    if k == 0:
                        av = [RX[k][(m + 3) & 3][3]] + RX[k][m & 3] + [RX[k][(m + 1) & 3][0]]
                    else:
                        av = [up((m + 1) & 3)[3]] + up((m + 2) & 3) + [up((m + 3) & 3)[0]]
                    for x in range(4):
                        vals = [bv[x + 2], bv[x + 1], bv[x], rgt[x], cen[x], left, av[x + 2], av[x + 1], av[x]]
                        a = w_desc[0] * vals[0]
                        for wq, v in zip(w_desc[1:], vals[1:]):
                            a = a + wq * v
                        out.append(a)
                        left = a
                outs.append(out)
            for k in range(32):
                g = tg + m - sk * k
                gin = 0 <= g < ng
                out = outs[k] if gin else [cval] * 4
                O[k][m & 3] = out
                if gin and 32 * b + k < n0:
                    for x in range(4):
                        u[32 * b + k, 4 * g + x] = out[x]
            for k in range(32):
                g = tg + m - sk * k
                RO[k][m & 3] = ld(32 * b + k, g + 4)
                RX[k][(m + qx0) & 3] = ld(xrow[k], g + lx) if k in (0, 31) else [cval] * 4
                RY[k][(m + qx0) & 3] = ld(yrow[k], g + lx) if k in (0, 31) and shape == "star2" else [cval] * 4


@pytest.mark.parametrize("ch", [8, 16, 32, 64])
@pytest.mark.parametrize("shape", ["star", "box", "star2"])
@pytest.mark.parametrize("n0,n1,T", [(40, 36, 3), (70, 12, 3), (33, 68, 2), (5, 8, 4)])
def test_random_orders_that_respect_the_waits_give_the_oracle_result(shape, n0, n1, T, ch):
    nb, ng, steps, order = geometry(n0, n1, T, ch, shape)
    nch = steps // ch
    cval = 0.3
    shp, r = ("star" if shape == "star2" else shape), radius(shape)
    w, u0 = case(2, shp, r, (n0, n1), seed=n0 + n1)
    w_desc = list(reversed(list(w)))
    ref = oracle_run(u0, T, 2, shp, r, w, "gs", "constant", cval, "unfused")
    rnd = inputs.uniform(4321 + n0, 100000)
    u = u0.reshape(n0, n1).copy()
    prog = {x: 0 for x in order}
    nxt = {x: 0 for x in order}
    states = {x: ([[None] * 4 for _ in range(32)], [[None] * 4 for _ in range(32)], [[None] * 4 for _ in range(32)],
                  [None] * 32) for x in order}
    pick = 0
    while True:
        ready = [x for x in order if nxt[x] < nch and
                 all(prog[y] >= need for y, need in chunk_waits(x[0], x[1], nxt[x] * ch, nb, ng, ch, shape))]
        if not ready:
            break
        x = ready[int(rnd[pick % len(rnd)] * len(ready))]
        pick += 1
        run_chunk(states[x], u, x[0], x[1], nxt[x], w_desc, cval, shape, n0, ng, ch)
        nxt[x] += 1
        prog[x] = nxt[x] * ch
    assert all(nxt[x] == nch for x in order), "the schedule stalled"
    got = u.reshape(u0.shape)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
