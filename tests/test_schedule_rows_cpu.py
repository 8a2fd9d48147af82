"""CPU restatement of the rows-as-lanes 2D Gauss-Seidel pipeline (k_gs2d_rows in csrc/k_wavefront.cu).

A task (s, b) is sweep s over band b (32 rows, one per lane); lane k updates column t - 2k at step t.
Each chunk of ch steps (32 by default, 64 or 128 when a plan asks) first waits for the progress of
(s, b-1), (s-1, b) and (s-1, b+1), then runs, then publishes. Every load a chunk issues (a lane's own row eight columns ahead, lane 0's row above and
lane 31's row below seven columns ahead, and the first chunk's ring fill) and every store is placed in
the chunk that issues it. The checks, on small ragged grids:
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

LAG = 62


def geometry(n0, n1, T, ch):
    nb = -(-n0 // 32)
    steps = -(-(n1 + LAG) // ch) * ch
    order = [(s, e - s) for e in range(T + nb - 1) for s in range(max(0, e - nb + 1), min(T - 1, e) + 1)]
    return nb, steps, order


def chunk_waits(s, b, t0, nb, n1, ch):
    """(task, progress needed) pairs a chunk starting at step t0 waits for (the kernel's nA, nO, nB)."""
    smax = n1 + LAG
    out = []
    nA, nO, nB = t0 + ch + 7 + LAG, t0 + ch + 8, t0 + ch - 55
    if b > 0:
        out.append(((s, b - 1), min(nA, smax)))
    if s > 0:
        out.append(((s - 1, b), min(nO, smax)))
    if s > 0 and b + 1 < nb and nB > 0:
        out.append(((s - 1, b + 1), min(nB, smax)))
    return out


def chunk_access(s, b, c, n0, n1, ch):
    """Points a chunk reads and writes."""
    rd, wr = set(), set()

    def add(row, col, into):
        if 0 <= row < n0 and 0 <= col < n1:
            into.add((row, col))
    t0 = c * ch
    if c == 0:
        for k in range(32):
            for q in range(8):
                add(32 * b + k, -2 * k + q, rd)
        for q in range(-1, 7):
            add(32 * b - 1, q, rd)
            add(32 * b + 32, -LAG + q, rd)
    for t in range(t0, t0 + ch):
        for k in range(32):
            j = t - 2 * k
            add(32 * b + k, j, wr)
            add(32 * b + k, j + 8, rd)
        add(32 * b - 1, t + 7, rd)
        add(32 * b + 32, t - LAG + 7, rd)
    return rd, wr


CASES = [(40, 37, 3), (64, 50, 3), (33, 70, 3), (5, 9, 4), (70, 13, 3), (70, 150, 3), (96, 40, 2), (1, 1, 2)]


@pytest.mark.parametrize("ch", [32, 64])
@pytest.mark.parametrize("n0,n1,T", CASES)
def test_waits_point_back_and_unordered_chunks_do_not_conflict(n0, n1, T, ch):
    nb, steps, order = geometry(n0, n1, T, ch)
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
        for (y, need) in chunk_waits(s, b, c * ch, nb, n1, ch):
            assert ticket[y] < ticket[(s, b)], "a wait names a later ticket"
            cy = -(-need // ch) - 1          # the chunk whose publication first reaches need
            assert 0 <= cy < nch
            p |= pred[idx[(y, cy)]] | (1 << idx[(y, cy)])
        pred[q] = p
        acc.append(chunk_access(s, b, c, n0, n1, ch))
    for a in range(len(inst)):
        ra, wa = acc[a]
        for bq in range(a + 1, len(inst)):
            if (pred[bq] >> a) & 1 or (pred[a] >> bq) & 1:
                continue
            rb, wb = acc[bq]
            assert not (wa & (rb | wb)), (inst[a], inst[bq])
            assert not (wb & ra), (inst[a], inst[bq])


def run_chunk(state, u, s, b, c, w_desc, cval, shape, n0, n1, ch):
    """One chunk of task (s, b), the lanes' registers emulated as the kernel holds them."""
    RO, RX, O = state

    def ld(row, col):
        return u[row, col] if 0 <= row < n0 and 0 <= col < n1 else cval
    xrow = [32 * b - 1 if k == 0 else 32 * b + 32 for k in range(32)]
    if c == 0:
        for k in range(32):
            for q in range(8):
                RO[k][q] = ld(32 * b + k, -2 * k + q)
            for q in range(-1, 7):
                RX[k][(q + 8) & 7] = ld(xrow[k], -2 * k + q) if k in (0, 31) else cval
            O[k] = [cval] * 4
    for tg in range(c * ch, c * ch + ch, 8):
        for m in range(8):
            outs = []
            for k in range(32):
                def dn(slot):      # __shfl_down_sync(RO[slot], 1); lane 31 keeps its own value
                    return RO[k + 1][slot] if k < 31 else RO[k][slot]

                def up(slot):      # __shfl_up_sync(O[slot], 1); lane 0 keeps its own value
                    return O[k - 1][slot] if k > 0 else O[k][slot]
                if shape == "star":
                    bel = RX[k][m & 7] if k == 31 else dn((m + 2) & 7)
                    abv = RX[k][m & 7] if k == 0 else up((m + 2) & 3)
                    vals = [bel, RO[k][(m + 1) & 7], RO[k][m & 7], O[k][(m + 3) & 3], abv]
                else:
                    if k == 31:
                        br, bc_, bl = RX[k][(m + 1) & 7], RX[k][m & 7], RX[k][(m + 7) & 7]
                    else:
                        br, bc_, bl = dn((m + 3) & 7), dn((m + 2) & 7), dn((m + 1) & 7)
                    if k == 0:
                        ar, ac, al = RX[k][(m + 1) & 7], RX[k][m & 7], RX[k][(m + 7) & 7]
                    else:
                        ar, ac, al = up((m + 3) & 3), up((m + 2) & 3), up((m + 1) & 3)
                    vals = [br, bc_, bl, RO[k][(m + 1) & 7], RO[k][m & 7], O[k][(m + 3) & 3], ar, ac, al]
                a = w_desc[0] * vals[0]
                for wq, v in zip(w_desc[1:], vals[1:]):
                    a = a + wq * v
                outs.append(a)
            for k in range(32):
                j = tg + m - 2 * k
                jin = 0 <= j < n1
                out = outs[k] if jin else cval
                O[k][m & 3] = out
                if jin and 32 * b + k < n0:
                    u[32 * b + k, j] = out
            for k in range(32):
                j = tg + m - 2 * k
                RO[k][m & 7] = ld(32 * b + k, j + 8)
                RX[k][(m + 7) & 7] = ld(xrow[k], j + 7) if k in (0, 31) else cval


@pytest.mark.parametrize("ch", [32, 64])
@pytest.mark.parametrize("shape", ["star", "box"])
@pytest.mark.parametrize("n0,n1,T", [(40, 37, 3), (70, 13, 3), (33, 70, 2), (5, 9, 4)])
def test_random_orders_that_respect_the_waits_give_the_oracle_result(shape, n0, n1, T, ch):
    nb, steps, order = geometry(n0, n1, T, ch)
    nch = steps // ch
    cval = 0.3
    w, u0 = case(2, shape, 1, (n0, n1), seed=n0 + n1)
    w_desc = list(reversed(list(w)))
    ref = oracle_run(u0, T, 2, shape, 1, w, "gs", "constant", cval, "unfused")
    rnd = inputs.uniform(4321 + n0, 100000)
    u = u0.reshape(n0, n1).copy()
    prog = {x: 0 for x in order}
    nxt = {x: 0 for x in order}
    states = {x: ([[0.0] * 8 for _ in range(32)], [[0.0] * 8 for _ in range(32)], [[0.0] * 4 for _ in range(32)])
              for x in order}
    pick = 0
    while True:
        ready = [x for x in order if nxt[x] < nch and
                 all(prog[y] >= need for y, need in chunk_waits(x[0], x[1], nxt[x] * ch, nb, n1, ch))]
        if not ready:
            break
        x = ready[int(rnd[pick % len(rnd)] * len(ready))]
        pick += 1
        run_chunk(states[x], u, x[0], x[1], nxt[x], w_desc, cval, shape, n0, n1, ch)
        nxt[x] += 1
        prog[x] = nxt[x] * ch
    assert all(nxt[x] == nch for x in order), "the schedule stalled"
    got = u.reshape(u0.shape)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
