"""CPU restatement of the periodic Gauss-Seidel tile DAG (k_gs_sweepdag in csrc/k_wavefront.cu).

Tiles of (lines along axes 0 and 1) x (hyperplane steps) are handed out in (sweep, diagonal) order;
a tile waits for its three lower neighbours of its own sweep and for the tiles of the previous sweep
that sweep_dag_prev_waits names. The checks, on small grids:
  * every wait names a tile instance with an earlier ticket (so the persistent kernel cannot
    deadlock: everything waited for was claimed earlier by a running CTA);
  * any two tile instances the waits leave unordered touch disjoint points: neither writes a point
    the other reads or writes;
  * executing the tiles in random orders that respect the waits gives the oracle's result, bit for
    bit (unfused rounding, which Python floats reproduce exactly).
Dropping any one of the three wrap rules makes the second check fail on some of these grids. The
first rule (the tile one radius beyond) is implied by the others for a periodic grid, through the
wrap waits of the tiles on the low faces that precede every tile; it is kept so that each tile's
previous-sweep dependences are covered by its own waits.
"""
import numpy as np
import pytest

from helpers import case, oracle_run
from paper_2010_04868_gb300 import inputs


def geometry(dim, ext, b0, b1, bs):
    n0, n1, n2 = [1] * (3 - dim) + list(ext)
    cp1 = 1
    cp0 = 1 if dim == 3 else 0
    b0 = b0 if dim == 3 else 1
    thmax = cp0 * (n0 - 1) + cp1 * (n1 - 1) + (n2 - 1)
    return dict(n0=n0, n1=n1, n2=n2, cp0=cp0, cp1=cp1, b0=b0, b1=b1, bs=bs,
                nt0=-(-n0 // b0), nt1=-(-n1 // b1), nts=thmax // bs + 1)


def prev_waits(t, dim, r, T0, T1, TS):
    """The previous sweep's tiles a tile waits for (a restatement of sweep_dag_prev_waits)."""
    def clamp(a, b, c):
        return (min(a, t["nt0"] - 1), min(b, t["nt1"] - 1), min(c, t["nts"] - 1))
    out = [clamp(T0 + -(-r // t["b0"]), T1 + -(-r // t["b1"]), TS + -(-r // t["bs"]))]
    i_lo, i_hi = T0 * t["b0"], min((T0 + 1) * t["b0"] - 1, t["n0"] - 1)
    j_lo, j_hi = T1 * t["b1"], min((T1 + 1) * t["b1"] - 1, t["n1"] - 1)
    th_lo, th_hi = TS * t["bs"], TS * t["bs"] + t["bs"] - 1
    if th_lo < t["cp0"] * i_hi + t["cp1"] * j_hi + r:
        out.append(clamp(T0, T1, (t["cp0"] * i_hi + t["cp1"] * j_hi + t["n2"] - 1) // t["bs"]))
    if j_lo < r:
        out.append(clamp(T0, t["nt1"] - 1, (t["cp1"] * (t["n1"] - 1) + th_hi) // t["bs"]))
    if dim == 3 and i_lo < r:
        out.append(clamp(t["nt0"] - 1, T1, (t["cp0"] * (t["n0"] - 1) + th_hi) // t["bs"]))
    return out


def tile_points(t, T0, T1, TS):
    """Points of a tile in execution order: hyperplane step by step."""
    pts = []
    for ls in range(t["bs"]):
        for l0 in range(t["b0"]):
            for l1 in range(t["b1"]):
                i = T0 * t["b0"] + l0
                j = T1 * t["b1"] + l1
                k = TS * t["bs"] + ls - t["cp0"] * i - t["cp1"] * j
                if i < t["n0"] and j < t["n1"] and 0 <= k < t["n2"]:
                    pts.append((i, j, k))
    return pts


def star_offsets(dim, r):
    offs = []
    for a in range(3 - dim, 3):
        for o in range(1, r + 1):
            for sgn in (-1, 1):
                d = [0, 0, 0]
                d[a] = sgn * o
                offs.append(tuple(d))
    return offs


def build(dim, ext, r, tiles, T):
    t = geometry(dim, ext, *tiles)
    n = (t["n0"], t["n1"], t["n2"])
    tl = [(a, b, c) for a in range(t["nt0"]) for b in range(t["nt1"]) for c in range(t["nts"])]
    # ticket order: sweep, then diagonal, then (T0, T1) as the kernel decodes it
    order = sorted(tl, key=lambda x: (x[0] + x[1] + x[2], x[0], x[1]))
    inst = [(s, x) for s in range(T) for x in order]
    ticket = {v: i for i, v in enumerate(inst)}
    offs = star_offsets(dim, r)
    reads, writes, waits = [], [], []
    for s, (T0, T1, TS) in inst:
        pts = tile_points(t, T0, T1, TS)
        wr = {p for p in pts}
        rd = set()
        for (i, j, k) in pts:
            for (a, b, c) in offs:
                rd.add(((i + a) % n[0], (j + b) % n[1], (k + c) % n[2]))
        w = []
        for d, x in ((0, (T0 - 1, T1, TS)), (1, (T0, T1 - 1, TS)), (2, (T0, T1, TS - 1))):
            if (T0, T1, TS)[d] > 0:
                w.append((s, x))
        if s > 0:
            w += [(s - 1, x) for x in prev_waits(t, dim, r, T0, T1, TS)]
        reads.append(rd)
        writes.append(wr)
        waits.append([ticket[v] for v in w])
    return t, inst, reads, writes, waits


CASES = [(3, (6, 7, 8), 1, (2, 2, 3)), (3, (5, 6, 7), 2, (1, 2, 2)), (3, (7, 5, 9), 1, (3, 2, 4)),
         (3, (5, 5, 5), 1, (4, 4, 2)), (2, (9, 10), 1, (1, 3, 4)), (2, (8, 11), 2, (1, 2, 3))]


@pytest.mark.parametrize("dim,ext,r,tiles", CASES)
def test_waits_point_back_and_unordered_tiles_do_not_conflict(dim, ext, r, tiles):
    t, inst, reads, writes, waits = build(dim, ext, r, tiles, T=3)
    m = len(inst)
    pred = [0] * m                       # bitset of transitive predecessors
    for q in range(m):
        for p in waits[q]:
            assert p < q, "a wait names a later ticket"
            pred[q] |= pred[p] | (1 << p)
    for a in range(m):
        for b in range(a + 1, m):
            if (pred[b] >> a) & 1:
                continue                  # a is ordered before b
            assert not (writes[a] & (reads[b] | writes[b])), (inst[a], inst[b])
            assert not (writes[b] & reads[a]), (inst[a], inst[b])


@pytest.mark.parametrize("dim,ext,r,tiles", CASES)
def test_random_orders_that_respect_the_waits_give_the_oracle_result(dim, ext, r, tiles):
    T = 3
    t, inst, reads, writes, waits = build(dim, ext, r, tiles, T)
    w, u0 = case(dim, "star", r, ext, seed=dim * 7 + r)
    canonical = sorted(star_offsets(dim, r) + [(0, 0, 0)])   # lexicographic, slowest axis first
    terms = list(reversed(list(zip(canonical, w))))    # descending canonical order
    ref = oracle_run(u0, T, dim, "star", r, w, "gs", "periodic", 0.0, "unfused")
    n = (t["n0"], t["n1"], t["n2"])
    rnd = inputs.uniform(1234 + dim, 100000)
    for trial in range(2):
        u = u0.reshape(n).copy()
        done = [False] * len(inst)
        left = len(inst)
        pick = 0
        while left:
            ready = [q for q in range(len(inst)) if not done[q] and all(done[p] for p in waits[q])]
            q = ready[int(rnd[(pick + trial * 5000) % len(rnd)] * len(ready))]
            pick += 1
            s, (T0, T1, TS) = inst[q]
            for (i, j, k) in tile_points(t, T0, T1, TS):
                acc = None
                for (a, b, c), wq in terms:
                    v = u[(i + a) % n[0], (j + b) % n[1], (k + c) % n[2]]
                    acc = wq * v if acc is None else acc + wq * v
                u[i, j, k] = acc
            done[q] = True
            left -= 1
        got = u.reshape(u0.shape)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
