"""CPU restatement of the streaming temporally blocked Jacobi kernel (csrc/k_stream.cu).

The emulation follows the kernel's geometry choice (make_str), its iteration structure (level-0
planes requested two iterations ahead, every level advancing M planes per iteration behind one
barrier), its ring slots and its per-level validity rules. Every ring cell carries a tag (level,
plane, iteration written); each read checks that it finds the plane it needs, written before the
last barrier and not yet overwritten, and that every index stays inside its ring. Every output
point must be written exactly once, and the result must equal the oracle bit for bit (unfused
rounding, which Python floats reproduce exactly).
"""
import itertools

import numpy as np
import pytest

from helpers import case, oracle_run


def canonical_offsets(dim, shape, r):
    offs = []
    r0 = range(-r, r + 1) if dim >= 3 else [0]
    r1 = range(-r, r + 1) if dim >= 2 else [0]
    for a in r0:
        for b in r1:
            for c in range(-r, r + 1):
                if shape == "star" and (a != 0) + (b != 0) + (c != 0) > 1:
                    continue
                offs.append((a, b, c))
    return offs


PF = 2   # iterations between requesting input planes and waiting for them


def stream_m(dim):
    return 4 if dim == 2 else 2


def make_str(dim, r, ext, tb, tile=(0, 0, 0), nsm=152, occ=3):
    """The kernel's launch geometry (a restatement of make_str in csrc/k_stream.cu)."""
    M = stream_m(dim)
    n0, n1, n2 = ([1] * (3 - dim) + list(ext))
    nz = n1 if dim == 2 else n0
    n1x = n1 if dim == 3 else 1
    h = tb * r
    pad = h & 1
    W2 = tile[2] if tile[2] > 0 else (256 if dim == 2 else 64)
    W2 = (W2 + 31) // 32 * 32
    W2 = min(W2, 256)
    while W2 - 2 * h - 2 * pad < 2 and W2 < 256:
        W2 += 32
    while W2 > 32 and W2 - 32 - 2 * h - 2 * pad >= n2:
        W2 -= 32
    B2 = W2 - 2 * h - 2 * pad
    if B2 < 2:
        return None
    if dim == 3:
        W1 = tile[1] if tile[1] > 0 else 16
        W1 = max(W1, 2 * h + 1)
        if W1 > 256:
            return None
        jg = 256 // W2
        W1 = (W1 + jg - 1) // jg * jg
        B1, J, block = W1 - 2 * h, W1 // jg, (W2, jg)
    else:
        W1, B1, J, block = 1, 1, 1, (W2, 1)
    C0 = ((PF + 2) * M + 2 * r + M - 1) // M * M
    C = 2 * M + 2 * r
    ns2 = (n2 + B2 - 1) // B2
    ns1 = (n1x + B1 - 1) // B1 if dim == 3 else 1
    total = ns1 * ns2 * nz
    per = tile[0] if tile[0] > 0 else (total + nsm * occ - 1) // (nsm * occ)
    per = max(per, 2 * M)
    nblk = (total + per - 1) // per
    planes = C0 + (tb - 1) * C
    smem = planes * W1 * W2 * 8
    if smem > 227 * 1024:
        return None
    return dict(M=M, W1=W1, W2=W2, B1=B1, B2=B2, h=h, pad=pad, J=J, block=block, C0=C0, C=C, per=per, ns1=ns1,
                ns2=ns2, nblk=nblk, smem=smem, nz=nz, n1=n1x, n2=n2)


def emulate(u0, dim, shape, r, w, bc, c, tb, tile=(0, 0, 0), tma=True):
    """One pass of tb steps as the kernel runs it; returns the output grid."""
    sg = make_str(dim, r, u0.shape, tb, tile)
    assert sg is not None
    M, W1, W2, h, pad, C0, C = sg["M"], sg["W1"], sg["W2"], sg["h"], sg["pad"], sg["C0"], sg["C"]
    nz, n1, n2 = sg["nz"], sg["n1"], sg["n2"]
    assert W2 % 32 == 0 and W2 <= 256 and W1 <= 256 and sg["block"][0] * sg["block"][1] <= 256
    u = u0.reshape(nz, n1, n2) if dim == 3 else u0.reshape(nz, 1, n2)
    out = np.full(u.shape, np.nan)
    written = np.zeros(u.shape, dtype=np.int64)
    offs = canonical_offsets(dim, shape, r)
    terms = list(reversed(list(zip(offs, w))))        # descending canonical order
    za = 1 if dim == 2 else 0
    constant = bc == "constant"
    total = sg["ns1"] * sg["ns2"] * nz
    OUTSIDE = -10 ** 15
    for b in range(sg["nblk"]):
        # rings of this CTA: values and tags (segment * 10^9 + plane, iteration from which readable)
        rings = [np.full((C0 if s == 0 else C, W1, W2), np.nan) for s in range(tb)]
        tag_row = [np.full((C0 if s == 0 else C, W1, W2), -10 ** 18, dtype=np.int64) for s in range(tb)]
        tag_ready = [np.full((C0 if s == 0 else C, W1, W2), 10 ** 9, dtype=np.int64) for s in range(tb)]
        pending = {}                                   # mbarrier -> load index in flight on it
        kbase, seg = 0, 0
        a, e = b * sg["per"], min(total, (b + 1) * sg["per"])
        assert a < e
        while a < e:
            t = a // nz
            z0 = a - t * nz
            z1 = min(nz, z0 + (e - a))
            t2, t1 = t % sg["ns2"], t // sg["ns2"]
            gj0 = t1 * sg["B1"] - h if dim == 3 else 0
            gx0 = t2 * sg["B2"] - h - pad
            if tma and constant:
                assert gx0 % 2 == 0 and -2 ** 31 <= gx0 < 2 ** 31   # TMA: x * 8 bytes on a 16-byte boundary
            gj = gj0 + np.arange(W1)[:, None] + np.zeros((1, W2), dtype=np.int64)
            gx = gx0 + np.arange(W2)[None, :] + np.zeros((W1, 1), dtype=np.int64)
            cell_out = (gx < 0) | (gx >= n2) | ((gj < 0) | (gj >= n1) if dim == 3 else False)
            c0 = z0 - tb * r
            niter = (z1 - z0 - 1 + 2 * tb * r + tb * M) // M + 1
            hi0 = z1 + tb * r
            tagbase = seg * 10 ** 9
            if constant:
                for s in range(1, tb):
                    rings[s][:, cell_out] = c
                    tag_row[s][:, cell_out] = OUTSIDE
                    tag_ready[s][:, cell_out] = 0

            def load(j, it_issue):
                k = kbase + j
                bar = k % (PF + 1)
                assert bar not in pending, "an mbarrier reused while its load is in flight"
                pending[bar] = k
                slot = (j * M) % C0
                assert slot + M <= C0
                for m in range(M):
                    z = c0 + j * M + m
                    if bc == "periodic":
                        vals = u[z % nz][(gj % n1), (gx % n2)]
                    else:
                        inside = (0 <= z < nz) & ~cell_out
                        vals = np.where(inside, u[min(max(z, 0), nz - 1)][np.clip(gj, 0, n1 - 1),
                                                                          np.clip(gx, 0, n2 - 1)], c)
                    rings[0][slot + m] = vals
                    tag_row[0][slot + m] = tagbase + z
                    tag_ready[0][slot + m] = j + 1
                assert it_issue == j - PF

            for j in range(PF):
                if j < niter and c0 + j * M < hi0:
                    load(j, j - PF)
            for it in range(niter):
                if it + PF < niter and c0 + (it + PF) * M < hi0:
                    load(it + PF, it)
                if c0 + it * M < hi0:
                    k = kbase + it
                    assert pending.pop(k % (PF + 1)) == k, "the wait finds the load it expects"
                for s in range(1, tb + 1):
                    cs = c0 - s * (M + r)
                    y0 = cs + it * M
                    lo, hi = z0 - (tb - s) * r, z1 + (tb - s) * r
                    if y0 + M <= lo or y0 >= hi:
                        continue
                    cin_base = c0 - (s - 1) * (M + r)
                    Cin = C0 if s == 1 else C
                    lo_col, hi_col = pad + s * r, pad + 2 * h + sg["B2"] - s * r
                    xs = np.arange(W2)
                    valid = (xs >= lo_col) & (xs < hi_col)
                    valid = np.broadcast_to(valid[None, :], (W1, W2)).copy()
                    if dim == 3:
                        js = np.arange(W1)
                        valid &= ((js >= s * r) & (js < W1 - s * r))[:, None]
                    if constant:
                        valid &= ~cell_out
                    acc = np.zeros((M, W1, W2))
                    for q, ((o0, o1, o2), wq) in enumerate(terms):
                        dz = (o0, o1, o2)[za]
                        dj = o1 if dim == 3 else 0
                        dx = o2
                        for m in range(M):
                            y = y0 + m + dz
                            slot = (y - cin_base) % Cin
                            jj = np.arange(W1)[:, None] + dj + np.zeros((1, W2), dtype=np.int64)
                            xx = np.arange(W2)[None, :] + dx + np.zeros((W1, 1), dtype=np.int64)
                            sel = valid & (lo <= y0 + m < hi)
                            if sel.any():
                                assert (jj[sel] >= 0).all() and (jj[sel] < W1).all()
                                assert (xx[sel] >= 0).all() and (xx[sel] < W2).all()
                                src_row = tag_row[s - 1][slot][jj[sel], xx[sel]]
                                src_ready = tag_ready[s - 1][slot][jj[sel], xx[sel]]
                                # outside cells: level 0 reloads them as c with every plane, higher levels
                                # hold c from the start of the segment
                                nb_out = (cell_out[jj[sel], xx[sel]] if (constant and s > 1)
                                          else np.zeros(sel.sum(), bool))
                                expect = np.where(nb_out, OUTSIDE, tagbase + y)
                                assert (src_row == expect).all(), (b, seg, s, it, y)
                                assert (src_ready <= it).all(), (b, seg, s, it, y)
                            v = rings[s - 1][slot][np.clip(jj, 0, W1 - 1), np.clip(xx, 0, W2 - 1)]
                            acc[m] = wq * v if q == 0 else acc[m] + wq * v
                    for m in range(M):
                        y = y0 + m
                        if y < lo or y >= hi:
                            continue
                        if s < tb:
                            slot = (it * M) % C + m
                            slot = slot - C if slot >= C else slot
                            assert slot == (y - cs) % C
                            val = c if (constant and (y < 0 or y >= nz)) else acc[m]
                            rings[s][slot][valid] = (val[valid] if isinstance(val, np.ndarray) else val)
                            tag_row[s][slot][valid] = tagbase + y
                            tag_ready[s][slot][valid] = it + 1
                        else:
                            lx = np.arange(W2) - pad - h
                            okx = (lx >= 0) & (lx < sg["B2"]) & (gx[0] < n2)
                            if dim == 3:
                                lj = np.arange(W1) - h
                                okj = (lj >= 0) & (lj < sg["B1"]) & (gj[:, 0] < n1)
                            else:
                                okj = np.array([True])
                            sel = valid & okx[None, :] & okj[:, None]
                            assert 0 <= y < nz
                            jj_g = gj[sel]
                            xx_g = gx[sel]
                            out[y, jj_g if dim == 3 else 0, xx_g] = acc[m][sel]
                            np.add.at(written[y], (jj_g if dim == 3 else np.zeros_like(xx_g), xx_g), 1)
            kbase += min(niter, -(-(hi0 - c0) // M))
            assert not pending, "every load of the segment was waited for"
            # the ring tags start from later iterations again in the next segment
            for s in range(tb):
                tag_ready[s][tag_ready[s] != 0] = -1
            a += z1 - z0
            seg += 1
    assert (written == 1).all(), "every output point written once"
    return out.reshape(u0.shape)


CASES = [
    # dim, shape, r, ext, bc, c, tb, tile
    (2, "star", 1, (37, 70), "constant", 0.0, 2, (0, 0, 32)),
    (2, "star", 1, (53, 301), "constant", 0.3, 4, (0, 0, 64)),
    (2, "box", 1, (40, 97), "constant", 0.25, 3, (9, 0, 64)),
    (2, "box", 1, (29, 66), "periodic", 0.0, 2, (7, 0, 32)),
    (2, "star", 2, (31, 90), "constant", 0.5, 2, (0, 0, 64)),
    (2, "box", 2, (26, 45), "periodic", 0.0, 1, (5, 0, 32)),
    (2, "star", 1, (5, 3), "constant", 0.1, 2, (0, 0, 0)),
    (3, "star", 1, (12, 11, 40), "constant", 0.2, 2, (5, 8, 32)),
    (3, "box", 1, (9, 10, 35), "periodic", 0.0, 2, (4, 6, 32)),
    (3, "star", 1, (7, 13, 70), "periodic", 0.0, 1, (0, 0, 64)),
    (3, "box", 1, (6, 5, 9), "constant", 0.0, 1, (0, 0, 0)),
]


@pytest.mark.parametrize("dim,shape,r,ext,bc,c,tb,tile", CASES)
def test_stream_schedule_and_result(dim, shape, r, ext, bc, c, tb, tile):
    if bc == "periodic" and min(ext) < 2 * r + 1:
        pytest.skip("periodic needs ext >= 2r+1")
    w, u0 = case(dim, shape, r, ext, seed=dim * 10 + tb)
    got = emulate(u0, dim, shape, r, list(w), bc, c, tb, tile)
    ref = oracle_run(u0, tb, dim, shape, r, w, "jacobi", bc, c, "unfused")
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


def test_default_geometry_of_the_4096_grid():
    """The default plan on the 4096^2 workload: 256-column strips, the planes shared out over one wave."""
    sg = make_str(2, 1, (4096, 4096), 2)
    assert sg["W2"] == 256 and sg["B2"] == 252 and sg["ns2"] == 17
    assert sg["nblk"] == 3 * 152 and sg["per"] * sg["nblk"] >= 17 * 4096 and sg["smem"] <= 227 * 1024
