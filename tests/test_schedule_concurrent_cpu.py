"""Schedules of the persistent kernels whose warps or CTAs wait on one
another, checked on the CPU before any GPU run.

k_jacobi_hex1d (split tiles, A and B segments of each period in one CTA, B
HEX_LAG levels behind A): each CTA is two coroutines, the compute warps (one
barrier per step) and the communication warp (releases this CTA's A levels,
acquires the next period's, fills a ring of 8 levels); the CTA barriers at band
ends join them. k_gs1d_wave4 (Gauss-Seidel sweeps on warp lanes, skew 33, one
chain warp and six partial-sum warps per 16-step batch): the warps' tasks of a
batch run in random order between barriers. k_gs2d_dec (2D 5-point
Gauss-Seidel, sweeps on warp lanes 3 rows apart, tiles of a DAG; per step the
chain warp's two newest-value terms and the producer warps' three
previous-sweep terms of the next step): tiles in random orders that respect
the DAG, the two roles of a step in either order, and every cell read checked
for the sweep its value must carry. Random interleavings of all coroutines
must neither deadlock nor read a value before it is published (every value
carries its band/level or step), and all must give the oracle's grid bit for
bit (unfused rounding).
"""
import random

import numpy as np
import pytest

from helpers import bits_equal, oracle_run
from paper_2010_04868_gb300 import inputs

HEX_LAG = 16


def run_hex1d(u0, T, r, w, bc, cval, H_req, n, seed):
    N, R, u = len(u0), r, u0.copy()
    H = min(H_req, (N // n) // (2 * R))
    fwA = fwB = 0
    for c in range(n):
        s0, s1 = c * N // n, (c + 1) * N // n
        W = min(s1 - s0, (s1 - s0 + 2 * H * R + 1) // 2)
        fwA, fwB = max(fwA, W + 2 * R), max(fwB, s1 - s0 - W + 2 * (H + 1) * R)
    flagA, flagB, aband, btop = [0] * n, [0] * n, {}, {}
    wd, od = list(reversed(w)), list(reversed(range(-R, R + 1)))
    clip, seqH = bc == "constant", H + 1

    def upd(src, i):
        vals = [src[i + o] for o in od]
        assert not any(np.isnan(v) for v in vals), "read unset"
        acc = wd[0] * vals[0]
        for q in range(1, len(vals)):
            acc = acc + wd[q] * vals[q]
        return acc

    class Cta:
        pass

    ctas = []
    for c in range(n):
        t = Cta()
        s0, s1 = c * N // n, (c + 1) * N // n
        W = min(s1 - s0, (s1 - s0 + 2 * H * R + 1) // 2)
        t.c, t.loA, t.hiA, t.loB, t.hiB = c, s0, s0 + W, s0 + W, s1
        t.hasL, t.hasR = (not clip) or c > 0, (not clip) or c < n - 1
        t.fA, t.fB = t.loA - R, t.loB - (H + 1) * R
        t.A = [np.full(fwA, np.nan), np.full(fwA, np.nan)]
        t.B = [np.full(fwB, np.nan), np.full(fwB, np.nan)]
        t.arb, t.alb, t.rvb = np.full(H * 2 * R, np.nan), {}, {}
        t.step_done = t.ring_ready = t.arrive = t.phase = 0
        ctas.append(t)

    def chk(i, fw):
        assert 0 <= i < fw, "frame index out of bounds"
        return i

    def bar0(t):
        gen = t.phase
        t.arrive += 1
        if t.arrive == 2:
            t.arrive, t.phase = 0, t.phase + 1
        while t.phase == gen:
            yield "wait"

    def compute(t):
        c, A, B, fA, fB = t.c, t.A, t.B, t.fA, t.fB
        for i in range(fwA):
            q = fA + i
            if q < 0 or q >= N:
                A[0][i] = A[1][i] = cval
            elif t.loA <= q < t.hiA:
                A[0][i] = u[q]
        for i in range(fwB):
            q = fB + i
            if clip and (q < 0 or q >= N):
                B[0][i] = B[1][i] = cval
            elif t.loB <= q < t.hiB:
                B[0][i] = u[q % N]
        g0 = done = b = 0
        while done < T:
            h = min(H, T - done)
            t.step_done = t.ring_ready = 0
            yield from bar0(t)
            for s in range(1, h + HEX_LAG + 1):
                kB, kx, kr = s - HEX_LAG, s - 1, s - HEX_LAG
                if s <= h:
                    L, U = t.loA + (s * R if t.hasL else 0), t.hiA - s * R
                    for i in range(L - fA, U - fA):
                        A[(g0 + s) & 1][chk(i, fwA)] = upd(A[(g0 + s - 1) & 1], i)
                if 1 <= kB <= h:
                    L, U = t.loB - kB * R, (min(t.hiB + kB * R, N) if clip else t.hiB + kB * R)
                    for i in range(L - fB, U - fB):
                        B[(g0 + kB) & 1][chk(i, fwB)] = upd(B[(g0 + kB - 1) & 1], i)
                if kx < h:
                    a = A[(g0 + kx) & 1]
                    for j in range(2 * R):
                        if t.hasL:
                            t.alb[(kx, j)] = (a[chk(t.loA + kx * R + j - fA, fwA)], b)
                        t.arb[kx * 2 * R + j] = a[chk(t.hiA - (kx + 2) * R + j - fA, fwA)]
                if 0 <= kr < h:
                    bb = B[(g0 + kr) & 1]
                    for j in range(2 * R):
                        bb[chk(t.loB - (kr + 2) * R + j - fB, fwB)] = t.arb[kr * 2 * R + j]
                    if t.hasR:
                        while t.ring_ready <= kr:
                            yield "wait ring"
                        for j in range(2 * R):
                            v, tag = t.rvb[(kr & 7, j)]
                            assert tag == (b, kr), "ring slot overwritten or stale"
                            bb[chk(t.hiB + kr * R + j - fB, fwB)] = v
                yield "step"
                t.step_done = s
            yield from bar0(t)
            bt, ab = B[(g0 + h) & 1], A[(g0 + h) & 1]
            if t.hasR:
                for i in range(h * R):
                    btop[(c, i)] = (bt[chk(t.hiB + i - fB, fwB)], b)
            for i in range(h * R):
                ab[chk(t.loB - h * R + i - fA, fwA)] = bt[chk(t.loB - h * R + i - fB, fwB)]
            yield from bar0(t)
            if t.hasR:
                flagB[c] = b + 1
            if t.hasL:
                while flagB[(c - 1) % n] < b + 1:
                    yield "wait B"
            yield from bar0(t)
            if t.hasL:
                for i in range(h * R):
                    v, vb = btop[((c - 1) % n, i)]
                    assert vb == b, "stale B top"
                    ab[chk(t.loA + i - fA, fwA)] = v
            done, g0, b = done + h, g0 + h, b + 1
        yield from bar0(t)
        for i in range(t.loA, t.hiA):
            u[i] = A[g0 & 1][i - fA]
        for i in range(t.loB, t.hiB):
            u[i] = B[g0 & 1][i - fB]

    def comm(t):
        c, cr = t.c, (t.c + 1) % n
        done = b = 0
        while done < T:
            h = min(H, T - done)
            yield from bar0(t)
            rel = lv = known = 0
            while (t.hasL and rel < h) or (t.hasR and lv < h):
                sd = t.step_done
                if t.hasL and rel < h and sd >= rel + 1:
                    upto = min(sd, h)
                    for k in range(rel, upto):
                        for j in range(2 * R):
                            v = t.alb[(k, j)]
                            assert v[1] == b, "staged band stale"
                            aband[(c, k, j)] = v
                    flagA[c] = max(flagA[c], b * seqH + upto)
                    rel = upto
                if t.hasR and lv < h and sd >= lv - 8 + HEX_LAG:
                    if known < b * seqH + lv + 1:
                        known = flagA[cr]
                    if known >= b * seqH + lv + 1:
                        last = min(known - b * seqH - 1, h - 1, sd + 8 - HEX_LAG)
                        for lvl in range(lv, last + 1):
                            for j in range(2 * R):
                                v, vb = aband[(cr, lvl, j)]
                                assert vb == b, "stale band of the next period"
                                t.rvb[(lvl & 7, j)] = (v, (b, lvl))
                        t.ring_ready, lv = last + 1, last + 1
                yield "comm"
            for _ in range(3):
                yield from bar0(t)
            done, b = done + h, b + 1
        yield from bar0(t)

    gens = {}
    for t in ctas:
        gens[(t.c, "c")], gens[(t.c, "m")] = compute(t), comm(t)
    rng, live, spins = random.Random(seed), set(gens), 0
    while live:
        k = rng.choice(sorted(live))
        try:
            ev = next(gens[k])
            spins = spins + 1 if ev.startswith("wait") else 0
            assert spins < 500000, "deadlock"
        except StopIteration:
            live.discard(k)
    return u


def run_gs1d_wave(u0, T, w, cval, seed, S=33, D=16):
    n, u = len(u0), u0.copy()
    wd, rng = list(reversed(w)), random.Random(seed)
    NS = 3
    for b in range((T + 31) // 32):  # blocks in ticket order: block b - 1 is complete when b reads its outputs
        L = min(32, T - 32 * b)
        O = [[None] * 32 for _ in range(NS * D)]
        Pb = [[[None] * 32 for _ in range(D)] for _ in range(2)]
        BOT = [None] * 64
        mmax = (n - 1 + S * (L - 1)) // D
        nw = [cval] * 32

        def bot_load(m):
            for i in range(32):
                x = D * m + i
                BOT[x % 64] = ((u[x] if 0 <= x < n else cval), x)

        def produce(m, ds):
            if m > mmax:
                return
            for d in ds:
                j = D * m + d
                for k in range(L):
                    x = j - S * k
                    if not 0 <= x < n:
                        continue
                    if k == 0:
                        v0, p0 = BOT[x % 64]
                        assert p0 == x, "lane 0 value not fetched"
                        v1 = cval
                        if x + 1 < n:
                            v1, p1 = BOT[(x + 1) % 64]
                            assert p1 == x + 1, "lane 0 value not fetched"
                    else:
                        e0, e1 = O[(j - S) % (NS * D)][k - 1], O[(j - S + 1) % (NS * D)][k - 1]
                        assert e0[1] == j - S and e1[1] == j - S + 1, "ring row overwritten or stale"
                        v0, v1 = e0[0], e1[0]
                    Pb[m & 1][d][k] = (wd[0] * v1 + wd[1] * v0, j)

        def chain(m):
            if m > mmax:
                return
            for k in range(32):
                for d in range(D):
                    j, x = D * m + d, D * m + d - S * k
                    if k < L and 0 <= x < n:
                        p, pj = Pb[m & 1][d][k]
                        assert pj == j, "partial sum stale"
                        nw[k] = p + wd[2] * nw[k]
                        O[j % (NS * D)][k] = (nw[k], j)
                    else:
                        O[j % (NS * D)][k] = (cval, j)

        def top_copy(m):
            if 0 <= m <= mmax:
                for d in range(D):
                    j = D * m + d
                    x = j - S * (L - 1)
                    if 0 <= x < n:
                        u[x] = O[j % (NS * D)][L - 1][0]

        bot_load(0)
        bot_load(1)
        produce(0, range(D))
        bot_load(2)
        for m in range(mmax + 2):
            tasks = [lambda: chain(m)] + [lambda ds=ds: produce(m + 1, ds) for ds in
                                         (range(0, 3), range(3, 6), range(6, 9), range(9, 12), range(12, 14),
                                          range(14, 16))] + [lambda: bot_load(m + 3), lambda: top_copy(m - 1)]
            rng.shuffle(tasks)  # the warps of a batch run concurrently: any order must do
            for f in tasks:
                f()
    return u


@pytest.mark.parametrize("N,r,bc,c,H,n", [(1000, 1, "constant", 0.6, 100, 5), (999, 1, "periodic", 0.0, 30, 6),
                                         (37, 1, "periodic", 0.0, 8, 1), (64, 2, "constant", 0.3, 5, 3),
                                         (300, 3, "periodic", 0.0, 9, 4)])
def test_concurrent_split_tiles_1d_schedule(N, r, bc, c, H, n):
    w = list(inputs.normalized_weights(N + r, 2 * r + 1))
    u0 = inputs.grid(N * 3 + r, (N,))
    for T in (H - 1 if H > 1 else 1, 2 * H + HEX_LAG):
        ref = oracle_run(u0, T, 1, "star", r, w, "jacobi", bc, c, "unfused")
        for seed in (1, 2):
            assert bits_equal(run_hex1d(u0, T, r, w, bc, c, H, n, seed), ref), (T, seed)


@pytest.mark.parametrize("N,T,c", [(1000, 70, 0.0), (77, 40, 0.5), (5, 33, 0.0), (1, 3, 0.7)])
def test_gauss_seidel_1d_wavefront_schedule(N, T, c):
    w = list(inputs.normalized_weights(N + 1, 3))
    u0 = inputs.grid(N + 9, (N,))
    ref = oracle_run(u0, T, 1, "star", 1, w, "gs", "constant", c, "unfused")
    for seed in (1, 2):
        assert bits_equal(run_gs1d_wave(u0, T, w, c, seed), ref), seed


def run_gs2d_dec(u0, T, w, cval, seed, H=16, W=16, S=3):
    """The decoupled 2D tile's schedule: lane k of sweep block b applies sweep 32 b + k + 1 at rows
    r0 + st (r0 = I H - S k) and columns p2 .. p2 + W - 1 (p2 = J W - k); the producers form the three
    previous-sweep terms of step st + 1 while the chain applies the two newest-value terms of step st."""
    n1, n2 = u0.shape
    u, ver = u0.copy(), np.zeros(u0.shape, dtype=np.int64)  # ver: sweeps applied to each cell
    wd, rng = list(reversed(w)), random.Random(seed)  # (+1,0), (0,+1), (0,0), (0,-1), (-1,0)
    R, L32, b1 = 1, 32, 1
    nI = -(-(n1 + S * (L32 - 1)) // H)
    nJ = -(-(n2 + b1 * (L32 - 1)) // W)
    nB = -(-T // 32)
    dI, dJ = (R + S * (L32 - 1)) // H + 2, (R + b1 * (L32 - 1)) // W + 2

    def deps(b, I, J):
        d = []
        if I > 0:
            d.append((b, I - 1, J))
        if J > 0:
            d.append((b, I, J - 1))
        if b > 0:
            d.append((b - 1, min(I + dI, nI - 1), min(J + dJ, nJ - 1)))
        return d

    def rd(q, col, sweeps):
        if not (0 <= q < n1 and 0 <= col < n2):
            return cval
        assert ver[q, col] == sweeps, ("cell read with the wrong sweep", q, col, ver[q, col], sweeps)
        return u[q, col]

    def tile(b, I, J):
        Lb = min(32, T - 32 * b)
        P, L0, A0 = [dict(), dict()], [dict(), dict()], {}
        above = [[cval] * W for _ in range(32)]

        def produce(sn):
            for k in range(Lb):
                q, p2, sw = I * H - S * k + sn, J * W - b1 * k, 32 * b + k
                if not 0 <= q < n1:
                    continue
                for m in range(W):
                    col = p2 + m
                    if 0 <= col < n2:
                        acc = wd[0] * rd(q + 1, col, sw)
                        acc = acc + wd[1] * rd(q, col + 1, sw)
                        P[sn & 1][(k, m)] = (acc + wd[2] * rd(q, col, sw), sn)
                    if sn == 0:
                        A0[(k, m)] = rd(q - 1, col, sw + 1) if q >= 1 and 0 <= col < n2 else cval
                L0[sn & 1][k] = (rd(q, p2 - 1, sw + 1), sn)

        def chain(st):
            for k in range(Lb):
                q, p2, sw = I * H - S * k + st, J * W - b1 * k, 32 * b + k
                if not 0 <= q < n1:
                    continue
                left, s0 = L0[st & 1][k]
                assert s0 == st, "newest left value stale"
                for m in range(W):
                    col = p2 + m
                    if 0 <= col < n2:
                        a = A0[(k, m)] if st == 0 else (cval if q == 0 else above[k][m])
                        p, sp = P[st & 1][(k, m)]
                        assert sp == st, "partial sum stale"
                        o = (p + wd[3] * left) + wd[4] * a
                        assert ver[q, col] == sw, "overwrites a value of the wrong sweep"
                        u[q, col], ver[q, col] = o, sw + 1
                        left = above[k][m] = o
                    else:
                        left = cval

        produce(0)
        for st in range(H):
            tasks = [lambda: chain(st)] + ([lambda: produce(st + 1)] if st + 1 < H else [])
            rng.shuffle(tasks)  # the chain and the producers of a step run concurrently
            for f in tasks:
                f()

    done, pending = set(), [(b, I, J) for b in range(nB) for I in range(nI) for J in range(nJ)]
    while pending:  # any order that respects the DAG
        ready = [t for t in pending if all(d in done for d in deps(*t))]
        assert ready, "the tile DAG deadlocks"
        t = ready[rng.randrange(len(ready))] if rng.random() < 0.7 else min(ready, key=lambda x: x[0] * 10 ** 6 +
                                                                                   (x[1] + x[2]))
        pending.remove(t)
        tile(*t)
        done.add(t)
    return u


@pytest.mark.parametrize("ext,T,c,H", [((20, 24), 40, 0.0, 16), ((37, 50), 70, 0.4, 16), ((9, 40), 33, 0.0, 4),
                                       ((1, 1), 3, 0.7, 16), ((40, 7), 35, 0.0, 8)])
def test_gauss_seidel_2d_decoupled_tile_schedule(ext, T, c, H):
    w = list(inputs.normalized_weights(ext[0] * 7 + T, 5))
    u0 = inputs.grid(ext[1] * 5 + T, ext)
    ref = oracle_run(u0, T, 2, "star", 1, w, "gs", "constant", c, "unfused")
    for seed in (1, 2):
        assert bits_equal(run_gs2d_dec(u0, T, w, c, seed, H=H), ref), seed
