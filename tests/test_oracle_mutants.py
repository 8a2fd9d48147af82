"""The pins catch plausible mistakes: each mutant of the C oracle must fail at least one.

Every mutant is a copy of stencil_oracle.c with one planted error (a dropped
term, a mirrored index, the wrong summation order or rounding mode, a wrong
boundary rule, a Gauss-Seidel sweep in the wrong order, ...), compiled on the
CPU into a temporary library and run through a quick subset of the pins.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2010_04868_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "stencil_oracle.c")

MUTANTS = {
    "ascending_order": [("int q = K - 1;", "int q = 0;"), ("for (q = K - 2; q >= 0; --q)", "for (q = 1; q < K; ++q)")],
    "drop_term": [("for (q = K - 2; q >= 0; --q)", "for (q = K - 2; q >= 1; --q)")],
    "mirror_slow_axis": [("i + off[3 * q]", "i - off[3 * q]")],
    "mirror_fast_axis": [("k + off[3 * q + 2]", "k - off[3 * q + 2]")],
    "gs_reverse_sweep": [("for (int64_t k = 0; k < g.n[2]; ++k)\n                        u[",
                          "for (int64_t k = g.n[2] - 1; k >= 0; --k)\n                        u[")],
    "periodic_as_constant": [("if (g->bc == OR_BC_PERIODIC) {", "if (0) {")],
    "halo_zero": [("return g->c;", "return 0.0;")],
    "fma_mode_unfused": [("acc = fma(wq, v, acc);", "acc = acc + wq * v;")],
    "unfused_mode_fused": [("double prod = wq * v;\n            acc = acc + prod;", "acc = fma(wq, v, acc);")],
    "jacobi_in_place": [("b[(i * g.n[1] + j) * g.n[2] + k] = update(a,", "a[(i * g.n[1] + j) * g.n[2] + k] = update(a,")],
    "star_has_corners": [("if (shape == OR_STAR && nz > 1) continue;", "if (shape == OR_STAR && nz > 2) continue;")],
    "field_point_shifted": [("* g->n[2] + k];", "* g->n[2] + (k + 1) % g->n[2]];")],
    "field_terms_swapped": [("return field[q * n +", "return field[(q == 0 ? 1 : (q == 1 ? 0 : q)) * n +")],
    "field_ignored": [("if (!field) return w[q];", "return w[q];")],
    "one_step_too_many": [("for (int64_t t = 0; t < T; ++t) {", "for (int64_t t = 0; t <= T; ++t) {")],
}


def _quick_pins(lib):
    """A fast subset of the pins; raises AssertionError/ValueError on the first mismatch."""
    def orc(u, T, **kw):
        return oracle.run(u, T, lib=lib, **kw)

    # P1: exact rationals
    for dim, ext, T in ((1, (9,), 3), (2, (5, 6), 2), (3, (3, 4, 3), 1)):
        offs = exact.canonical_offsets(dim, "star", 1)
        m = (inputs.splitmix64(40 + dim, 0, len(offs)) % np.uint64(3) + np.uint64(1)).astype(np.float64)
        w = m / 2.0 ** np.ceil(np.log2(m.sum()))
        u0 = inputs.dyadic_grid(50 + dim, ext, bits=4)
        for method, mname in ((oracle.JACOBI, "jacobi"), (oracle.GAUSS_SEIDEL, "gs")):
            for bc, bname in ((oracle.BC_CONSTANT, "constant"), (oracle.BC_PERIODIC, "periodic")):
                TT = 1 if (mname == "gs" and bname == "periodic") else T
                ref = exact.to_array(exact.run(u0, TT, dim=dim, shape="star", r=1, weights=w, method=mname,
                                               bc=bname, c=0.375, require_representable=True), ext)
                for arith in (oracle.ARITH_FMA, oracle.ARITH_UNFUSED):
                    got = orc(u0, TT, dim=dim, shape=oracle.STAR, r=1, weights=w, method=method, bc=bc,
                              c=0.375, arith=arith)
                    assert np.array_equal(got, ref), ("P1", dim, mname, bname, arith)
    # P1b: rounding emulation
    w = inputs.normalized_weights(103, 5)
    u0 = inputs.grid(204, (5, 6))
    for mname, method in (("jacobi", oracle.JACOBI), ("gs", oracle.GAUSS_SEIDEL)):
        for rounding, arith in (("fma", oracle.ARITH_FMA), ("unfused", oracle.ARITH_UNFUSED)):
            ref = exact.to_array(exact.run(u0, 2, dim=2, shape="star", r=1, weights=w, method=mname,
                                           c=0.1, rounding=rounding), (5, 6))
            got = orc(u0, 2, dim=2, shape=oracle.STAR, r=1, weights=w, method=method, c=0.1, arith=arith)
            assert np.array_equal(got, ref), ("P1b", mname, rounding)
    # per-point weights: rounding emulation with a coefficient field
    for dim, shape, ext in ((2, "box", (4, 5)), (3, "star", (3, 4, 4))):
        k = len(exact.canonical_offsets(dim, shape, 1))
        field = inputs.uniform(60 + dim, k * int(np.prod(ext))).reshape((k,) + ext) / k
        u0 = inputs.grid(61 + dim, ext)
        for mname, method in (("jacobi", oracle.JACOBI), ("gs", oracle.GAUSS_SEIDEL)):
            ref = exact.to_array(exact.run(u0, 2, dim=dim, shape=shape, r=1, weights=[0.0] * k, method=mname,
                                           c=0.3, rounding="fma", field=field), ext)
            got = orc(u0, 2, dim=dim, shape=oracle.STAR if shape == "star" else oracle.BOX, r=1,
                      weights=[0.0] * k, method=method, c=0.3, field=field)
            assert np.array_equal(got, ref), ("field", dim, mname)
    # P2: Fourier decay, periodic Jacobi
    ext = (16, 24)
    offs = exact.canonical_offsets(2, "box", 1)
    w = inputs.normalized_weights(302, len(offs))
    theta = np.array([2 * np.pi / 16, 4 * np.pi / 24])
    idx = np.indices(ext)
    phase = theta[0] * idx[0] + theta[1] * idx[1]
    lam = sum(wi * np.exp(1j * np.dot(theta, o)) for wi, o in zip(w, offs))
    got = orc(np.cos(phase), 10, dim=2, shape=oracle.BOX, r=1, weights=w, bc=oracle.BC_PERIODIC)
    assert np.max(np.abs(got - np.real(lam ** 10 * np.exp(1j * phase)))) < 1e-13, "P2"
    # P4: constant field with halo c
    w = np.array([1, 1, 28, 1, 1]) / 32.0
    for method in (oracle.JACOBI, oracle.GAUSS_SEIDEL):
        got = orc(np.full((7, 6), 0.8125), 5, dim=2, shape=oracle.STAR, r=1, weights=w, method=method, c=0.8125)
        assert np.all(got == 0.8125), "P4"


def _build_variant(tmp_path, name, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert old in src, (name, old)
        src = src.replace(old, new)
    c = tmp_path / (name + ".c")
    c.write_text(src)
    so = tmp_path / (name + ".so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(c),
                           "-lm"])
    return oracle.load(str(so))


def test_unmutated_oracle_passes_quick_pins(tmp_path):
    _quick_pins(_build_variant(tmp_path, "original", []))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    lib = _build_variant(tmp_path, name, MUTANTS[name])
    with pytest.raises((AssertionError, ValueError)):
        _quick_pins(lib)
