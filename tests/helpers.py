"""Shared helpers for the tests: run a stencil through the C ABI and through the oracle."""
import numpy as np

import oracle
from paper_2010_04868_gb300 import inputs

SHAPE_ID = {"star": 0, "box": 1}
BC_ID = {"constant": 0, "periodic": 1}
METHOD_ID = {"jacobi": 0, "gs": 1}
ARITH_ID = {"fma": 0, "unfused": 1}


def k_of(dim, shape, r):
    return 2 * dim * r + 1 if (shape == "star" or dim == 1) else (2 * r + 1) ** dim


def case(dim, shape, r, ext, seed=1, weights="normalized"):
    k = k_of(dim, shape, r)
    w = inputs.normalized_weights(seed * 7 + 3, k)
    u0 = inputs.grid(seed, ext)
    return w, u0


def oracle_run(u0, T, dim, shape, r, w, method, bc, c, arith):
    return oracle.run(u0, T, dim=dim, shape=SHAPE_ID[shape] if dim > 1 else 0, r=r, weights=w,
                      method=METHOD_ID[method], bc=BC_ID[bc], c=c, arith=ARITH_ID[arith])


def gpu_run(u0, T, dim, shape, r, w, method, bc, c, arith, plan=None, tb=0, tile=(0, 0, 0), use_scratch=True):
    import torch
    from paper_2010_04868_gb300 import stencil as S
    st = S.Stencil(dim, SHAPE_ID[shape], r, list(w), METHOD_ID[method], BC_ID[bc], c, ARITH_ID[arith])
    if plan is not None:
        st.set_plan(plan, tb, tile)
    u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    scratch = torch.empty_like(u) if (use_scratch and method == "jacobi") else None
    st.run(u, T, scratch)
    rc = st.status()
    assert rc == 0, S.strerror(rc)
    torch.cuda.synchronize()
    out = u.cpu().numpy()
    st.close()
    return out


def bits_equal(a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


def first_diff(a, b):
    d = np.argwhere(a.view(np.uint64) != b.view(np.uint64))
    if len(d) == 0:
        return None
    idx = tuple(d[0])
    return idx, a[idx], b[idx], len(d)
