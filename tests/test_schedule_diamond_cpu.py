"""The split (diamond) tiling's schedule, checked on the CPU before any GPU run.

A plain-Python restatement of k_jacobi_diamond's index arithmetic: periods and
A/B segments per axis, the frame of each tile in shared memory, the per-level
edge bands in the workspace, the ring of level k fetched three levels ahead
(cp.async), and the 2^d phases of a band in lexicographic order. Buffers start
as NaN and band entries carry the band they were written in, so a read of a
value that was never written, or of a stale one, fails; every frame and band
index is bounds-checked; the ring copies land either at once or at the last
moment the kernel allows (its cp.async.wait_group), and both orders must give
the oracle's grid bit for bit (unfused rounding, which plain Python floats do
exactly).
"""
import itertools

import numpy as np
import pytest

from helpers import bits_equal, case, oracle_run

AHEAD = 4  # ring fetches in flight: the ring of level k is requested at level k - AHEAD + 1


def geometry(dim, r, N, H, P_in, nsm=152):
    act = [d >= 3 - dim for d in range(3)]
    P = list(P_in)
    n = [1, 1, 1]
    for d in range(3):
        if not act[d]:
            P[d] = 1
            continue
        if P[d] <= 0:
            P[d] = {1: max((N[d] + 4 * nsm - 1) // (4 * nsm), 64 * r), 2: 88, 3: 24}[dim]
        P[d] = max(P[d], 2 * r)
    pmin = 10 ** 18
    for d in range(3):
        if act[d]:
            n[d] = max(1, N[d] // P[d])
            pmin = min(pmin, N[d] // n[d])
    H = min(H, pmin // (2 * r))
    assert H >= 1
    fw = [1, 1, 1]
    for d in range(3):
        if act[d]:
            for c in range(n[d]):
                s0, s1 = c * N[d] // n[d], (c + 1) * N[d] // n[d]
                W = min(s1 - s0, (s1 - s0 + 2 * H * r + 1) // 2)
                fw[d] = max(fw[d], W + 2 * r, s1 - s0 - W + 2 * (H + 1) * r)
    other = [N[0] * N[1] * N[2] // N[d] for d in range(3)]
    return act, n, H, fw, other


def run_split(u0, T, dim, shape, r, w, bc, cval, H_req, P_in, late):
    N = [1, 1, 1]
    for d in range(dim):
        N[3 - dim + d] = u0.shape[d]
    act, n, H, fw, other = geometry(dim, r, N, H_req, P_in)
    F = fw[0] * fw[1] * fw[2]
    u = u0.reshape(-1).copy()
    band = [dict() for _ in range(3)]
    rng_off = range(-r, r + 1)
    offs = [(a, b, c) for a in (rng_off if dim >= 3 else [0]) for b in (rng_off if dim >= 2 else [0]) for c in rng_off
            if shape == "box" or (a != 0) + (b != 0) + (c != 0) <= 1]
    wd, od = list(reversed(w)), list(reversed(offs))

    def inb(q):
        return all(0 <= q[d] < N[d] for d in range(3))

    def gidx(q):
        q = [q[d] % N[d] for d in range(3)]
        return (q[0] * N[1] + q[1]) * N[2] + q[2]

    def oth(d, q):
        q = [q[e] % N[e] for e in range(3)]
        return q[1] * N[2] + q[2] if d == 0 else (q[0] * N[2] + q[2] if d == 1 else q[0] * N[1] + q[1])

    def bkey(d, k, e, j, o):
        assert 0 <= k < H and 0 <= e < 2 * n[d] and 0 <= j < 2 * r and 0 <= o < other[d]
        return (k, e, j, o)

    phases = [m for m in range(8) if all(not ((m >> (2 - d)) & 1) or act[d] for d in range(3))]
    done, bno = 0, 0
    while done < T:
        h = min(H, T - done)
        for ph in phases:
            for tc in itertools.product(*[range(n[d]) for d in range(3)]):
                lo, hi, f0, isB, shL = [0] * 3, [1] * 3, [0] * 3, [0] * 3, [0] * 3
                for d in range(3):
                    if not act[d]:
                        continue
                    s0, s1 = tc[d] * N[d] // n[d], (tc[d] + 1) * N[d] // n[d]
                    W = min(s1 - s0, (s1 - s0 + 2 * H * r + 1) // 2)
                    isB[d] = (ph >> (2 - d)) & 1
                    if not isB[d]:
                        lo[d], hi[d], f0[d] = s0, s0 + W, s0 - r
                        shL[d] = int(bc == "periodic" or s0 > 0)
                    else:
                        lo[d], hi[d], f0[d], shL[d] = s0 + W, s1, s0 + W - (H + 1) * r, 1

                def region(d, k):
                    if not act[d]:
                        return 0, 1
                    if not isB[d]:
                        return lo[d] + (k * r if shL[d] else 0), hi[d] - k * r
                    L, U = lo[d] - k * r, hi[d] + k * r
                    return L, (min(U, N[d]) if bc == "constant" else U)

                def fpos(q):
                    p = [q[d] - f0[d] for d in range(3)]
                    assert all(0 <= p[d] < fw[d] for d in range(3)), "frame index out of bounds"
                    return (p[0] * fw[1] + p[1]) * fw[2] + p[2]

                buf = [np.full(F, np.nan), np.full(F, np.nan)]
                if bc == "constant":
                    for i in range(F):
                        q = (f0[0] + i // (fw[1] * fw[2]), f0[1] + (i // fw[2]) % fw[1], f0[2] + i % fw[2])
                        if not inb(q):
                            buf[0][i] = buf[1][i] = cval
                R0 = [region(d, 0) for d in range(3)]
                for q in itertools.product(*[range(*R0[d]) for d in range(3)]):
                    buf[0][fpos(q)] = u[gidx(q)]

                def ring_writes(k):
                    """The ring of level k: (frame position, value) pairs, read from the bands."""
                    out = []
                    Rk = [region(d, k) for d in range(3)]
                    for d in range(3):
                        if not act[d] or not isB[d]:
                            continue
                        lo2 = [Rk[a][0] - (2 * r if a > d and act[a] and isB[a] else 0) for a in range(3)]
                        hi2 = [Rk[a][1] + (2 * r if a > d and act[a] and isB[a] else 0) for a in range(3)]
                        for jj in range(4 * r):
                            for qa in itertools.product(*[range(lo2[a], hi2[a]) if a != d else [0] for a in range(3)]):
                                q = list(qa)
                                if jj < 2 * r:
                                    q[d], e, j = Rk[d][0] - 2 * r + jj, 2 * tc[d] + 1, jj
                                else:
                                    q[d], e, j = hi[d] + k * r + jj - 2 * r, 2 * ((tc[d] + 1) % n[d]), jj - 2 * r
                                if bc == "constant" and not inb(q):
                                    continue
                                v, vb = band[d][bkey(d, k, e, j, oth(d, q))]
                                assert vb == bno, "stale band value"
                                out.append((fpos(q), v))
                    return out

                def export(k, b):
                    Rk = [region(d, k) for d in range(3)]
                    for d in range(3):
                        if not act[d] or isB[d]:
                            continue
                        for side in ([0, 1] if shL[d] else [1]):
                            start = Rk[d][0] if side == 0 else Rk[d][1] - 2 * r
                            for j in range(2 * r):
                                for qa in itertools.product(*[range(*Rk[a]) if a != d else [0] for a in range(3)]):
                                    q = list(qa)
                                    q[d] = start + j
                                    v = b[fpos(q)]
                                    assert not np.isnan(v), "export of an unset value"
                                    band[d][bkey(d, k, 2 * tc[d] + side, j, oth(d, q))] = (v, bno)

                pending = []  # groups of ring writes in flight: (buffer, writes)

                def commit(k):
                    g = (buf[k & 1], ring_writes(k)) if k < h else (None, [])
                    if late:
                        pending.append(g)
                    else:
                        for i, v in g[1]:
                            g[0][i] = v

                def wait(nkeep):
                    while len(pending) > nkeep:
                        b, ws = pending.pop(0)
                        for i, v in ws:
                            b[i] = v

                for k in range(AHEAD):
                    commit(k)
                wait(AHEAD - 1)
                for k in range(1, h + 1):
                    src, dst = buf[(k - 1) & 1], buf[k & 1]
                    export(k - 1, src)
                    commit(k + AHEAD - 1)
                    Rk = [region(d, k) for d in range(3)]
                    for q in itertools.product(*[range(*Rk[d]) for d in range(3)]):
                        dst[fpos(q)] = np.nan  # a level is never read before it is computed
                    for q in itertools.product(*[range(*Rk[d]) for d in range(3)]):
                        vals = [src[fpos((q[0] + o[0], q[1] + o[1], q[2] + o[2]))] for o in od]
                        assert not any(np.isnan(v) for v in vals), "read of a value not yet computed or fetched"
                        acc = wd[0] * vals[0]
                        for qq in range(1, len(vals)):
                            acc = acc + wd[qq] * vals[qq]
                        dst[fpos(q)] = acc
                    wait(AHEAD - 1)
                wait(0)
                Rh = [region(d, h) for d in range(3)]
                for q in itertools.product(*[range(*Rh[d]) for d in range(3)]):
                    u[gidx(q)] = buf[h & 1][fpos(q)]
        done += h
        bno += 1
    return u.reshape(u0.shape)


CASES = [(1, "star", 1, (37,), 4, (0, 0, 10)), (1, "star", 2, (301,), 5, (0, 0, 37)),
         (2, "star", 1, (30, 58), 4, (0, 12, 17)), (2, "box", 1, (20, 26), 3, (0, 9, 8)),
         (3, "star", 1, (10, 7, 9), 1, (3, 3, 4)), (3, "box", 1, (9, 8, 12), 2, (4, 4, 5))]


@pytest.mark.parametrize("dim,shape,r,ext,H,periods", CASES)
@pytest.mark.parametrize("bc,c", [("constant", 0.7), ("periodic", 0.0)])
def test_split_tiling_schedule(dim, shape, r, ext, H, periods, bc, c):
    if bc == "periodic" and min(ext) < 2 * r + 1:
        pytest.skip("periodic needs ext >= 2r+1")
    w, u0 = case(dim, shape, r, ext, seed=3)
    for T in (1, H + 1, 2 * H + 3):
        ref = oracle_run(u0, T, dim, shape, r, w, "jacobi", bc, c, "unfused")
        for late in (False, True):
            assert bits_equal(run_split(u0, T, dim, shape, r, w, bc, c, H, periods, late), ref), (T, late)
