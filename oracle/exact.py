"""Exact-rational restatement of the stencil definition (TEST INFRASTRUCTURE ONLY).

A third, independent code for the same definition as ``stencil_oracle.c``
(naive loops, Section 1 / Algorithm 1; in-place lexicographic Gauss-Seidel,
Section 3.4), in pure Python over ``fractions.Fraction``. Used to pin the C
oracle on tiny grids:

* ``rounding=None``: exact arithmetic, no rounding anywhere. With dyadic
  weights and inputs whose results stay exactly representable, the float
  oracle must agree bit for bit.
* ``rounding="fma"`` / ``"unfused"``: every operation is done exactly and
  then rounded to the nearest float64 (ties to even) with ``float(Fraction)``,
  which Python performs correctly rounded. This emulates the two rounding
  modes without relying on C's fma() or on compiler contraction flags.

Offsets are generated here independently of the C code, in the canonical
order (lexicographic, slowest dimension first, components -r..r).
"""
from __future__ import annotations

import itertools
from fractions import Fraction


def canonical_offsets(dim: int, shape: str, r: int):
    offs = []
    for o in itertools.product(range(-r, r + 1), repeat=dim):
        if shape == "star" and sum(1 for v in o if v != 0) > 1:
            continue
        offs.append(o)
    return offs


def _rnd(x: Fraction) -> Fraction:
    return Fraction(float(x))


def run(u, T, *, dim, shape, r, weights, method="jacobi", bc="constant", c=0.0, rounding=None,
        require_representable=False, field=None):
    """u: nested lists or numpy array; returns a dict {index tuple: Fraction}.

    require_representable: with rounding=None, raise ArithmeticError if any
    product or partial sum is not exactly a float64 (the case is then unfit
    for a bit-exact comparison with a float implementation).
    field: optional per-point weights, array of shape (K,) + grid shape in
    canonical term order; the weight of term q at point p is field[q][p].
    """
    import numpy as np

    arr = np.asarray(u, dtype=np.float64)
    ext = arr.shape
    offs = canonical_offsets(dim, shape, r)
    assert len(offs) == len(weights)
    W = [Fraction(float(w)) for w in weights]
    F = None if field is None else np.asarray(field, dtype=np.float64)

    def wt(q, p):
        return W[q] if F is None else Fraction(float(F[(q,) + tuple(p)]))
    C = Fraction(float(c))
    pts = list(itertools.product(*[range(n) for n in ext]))   # lexicographic order
    cur = {p: Fraction(float(arr[p])) for p in pts}

    def get(state, q):
        if bc == "periodic":
            q = tuple(qi % n for qi, n in zip(q, ext))
            return state[q]
        if all(0 <= qi < n for qi, n in zip(q, ext)):
            return state[q]
        return C

    def point(state, p):
        order = list(range(len(offs) - 1, -1, -1))      # descending canonical order
        q0 = order[0]
        acc = wt(q0, p) * get(state, tuple(pi + oi for pi, oi in zip(p, offs[q0])))
        if rounding is not None:
            acc = _rnd(acc)
        elif require_representable and _rnd(acc) != acc:
            raise ArithmeticError("product not representable")
        for q in order[1:]:
            v = get(state, tuple(pi + oi for pi, oi in zip(p, offs[q])))
            if rounding is None:
                prod = wt(q, p) * v
                acc = acc + prod
                if require_representable and (_rnd(prod) != prod or _rnd(acc) != acc):
                    raise ArithmeticError("intermediate not representable")
            elif rounding == "fma":
                acc = _rnd(wt(q, p) * v + acc)
            else:
                acc = _rnd(acc + _rnd(wt(q, p) * v))
        return acc

    for _ in range(T):
        if method == "jacobi":
            cur = {p: point(cur, p) for p in pts}
        else:
            for p in pts:
                cur[p] = point(cur, p)
    return cur


def to_array(state, ext):
    import numpy as np

    out = np.empty(ext, dtype=np.float64)
    for p, v in state.items():
        out[p] = float(v)
    return out
