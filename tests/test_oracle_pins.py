"""Pins for the CPU oracle: checks against what the mathematics fixes.

Each test ties the C oracle to something other than itself:
  P1  exact rationals on tiny grids (dyadic data, results exactly representable)
  P1b IEEE rounding emulated with exact rationals (term order + rounding mode)
  P2  Fourier-mode decay for periodic Jacobi (closed form)
  P3  Dirichlet sine-mode decay for symmetric Jacobi (closed form)
  P4  constant-field invariance
  P5  identity and shift special cases
  P6  Gauss-Seidel equals Jacobi when no newest-value term has weight
  P7  Young's theorem: Gauss-Seidel asymptotic decay rate
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2010_04868_gb300 import inputs

EPS = 2.0 ** -53
SHAPES = {"star": oracle.STAR, "box": oracle.BOX}
METHODS = {"jacobi": oracle.JACOBI, "gs": oracle.GAUSS_SEIDEL}
BCS = {"constant": oracle.BC_CONSTANT, "periodic": oracle.BC_PERIODIC}


def dyadic_weights(offs, seed):
    """Non-symmetric dyadic weights m/2^b (m in 1..3), scaled so that they sum to <= 1.

    Few fraction bits per operation keep every intermediate exactly
    representable on tiny grids (checked by require_representable).
    """
    k = len(offs)
    m = inputs.splitmix64(seed, 0, k) % np.uint64(3) + np.uint64(1)
    m = m.astype(np.float64)
    b = math.ceil(math.log2(m.sum()))
    return m / 2.0 ** b


CASES = [
    # dim, shape, r, ext, T
    (1, "star", 1, (9,), 3),
    (1, "star", 2, (8,), 2),
    (2, "star", 1, (5, 6), 2),
    (2, "box", 1, (4, 5), 1),
    (2, "star", 2, (5, 5), 1),
    (3, "star", 1, (3, 4, 3), 1),
    (3, "box", 1, (3, 3, 3), 1),
]


@pytest.mark.parametrize("dim,shape,r,ext,T", CASES)
@pytest.mark.parametrize("method", ["jacobi", "gs"])
@pytest.mark.parametrize("bc", ["constant", "periodic"])
def test_p1_exact_rationals(dim, shape, r, ext, T, method, bc):
    if bc == "periodic" and min(ext) < 2 * r + 1:
        pytest.skip("periodic needs ext >= 2r+1")
    if shape == "box" and method == "gs" and (dim == 3 or bc == "periodic"):
        pytest.skip("the Gauss-Seidel chain outgrows 53 bits here; covered by P1b")
    if method == "gs" and bc == "periodic":
        T = 1          # the wrap chains whole sweeps together; one sweep keeps the chain short
    offs = exact.canonical_offsets(dim, shape, r)
    w = dyadic_weights(offs, 11 + dim * 7 + r)
    u0 = inputs.dyadic_grid(5 + dim, ext, bits=4)
    c = 0.375
    ref = exact.to_array(exact.run(u0, T, dim=dim, shape=shape, r=r, weights=w, method=method, bc=bc, c=c,
                                   require_representable=True), ext)
    for arith in (oracle.ARITH_FMA, oracle.ARITH_UNFUSED):
        got = oracle.run(u0, T, dim=dim, shape=SHAPES[shape], r=r, weights=w, method=METHODS[method],
                         bc=BCS[bc], c=c, arith=arith)
        assert np.array_equal(got, ref), (arith, np.max(np.abs(got - ref)))


@pytest.mark.parametrize("dim,shape,r,ext,T", [
    (1, "star", 1, (9,), 4), (2, "star", 1, (5, 6), 2), (2, "box", 1, (4, 5), 2), (3, "star", 1, (3, 4, 4), 1),
    (3, "box", 1, (3, 3, 4), 1), (1, "star", 3, (8,), 2)])
@pytest.mark.parametrize("method", ["jacobi", "gs"])
@pytest.mark.parametrize("rounding", ["fma", "unfused"])
@pytest.mark.parametrize("bc", ["constant", "periodic"])
def test_p1b_rounding_emulated(dim, shape, r, ext, T, method, rounding, bc):
    """Random (non-dyadic) data: every rounding of the chosen order and mode is reproduced."""
    if bc == "periodic" and min(ext) < 2 * r + 1:
        pytest.skip("periodic needs ext >= 2r+1")
    offs = exact.canonical_offsets(dim, shape, r)
    w = inputs.normalized_weights(101 + dim, len(offs))
    u0 = inputs.grid(202 + dim, ext)
    ref = exact.to_array(exact.run(u0, T, dim=dim, shape=shape, r=r, weights=w, method=method,
                                   bc=bc, c=0.1, rounding=rounding), ext)
    arith = oracle.ARITH_FMA if rounding == "fma" else oracle.ARITH_UNFUSED
    got = oracle.run(u0, T, dim=dim, shape=SHAPES[shape], r=r, weights=w, method=METHODS[method],
                     bc=BCS[bc], c=0.1, arith=arith)
    assert np.array_equal(got, ref)


def test_p1b_modes_and_order_are_distinguishable():
    """The two modes and the descending order are observable on random data (else P1b pins nothing)."""
    w = inputs.normalized_weights(7, 5)
    u0 = inputs.grid(8, (6, 7))
    a = oracle.run(u0, 3, dim=2, shape=oracle.STAR, r=1, weights=w, arith=oracle.ARITH_FMA)
    b = oracle.run(u0, 3, dim=2, shape=oracle.STAR, r=1, weights=w, arith=oracle.ARITH_UNFUSED)
    assert not np.array_equal(a, b)
    # reversing the coefficient list and mirroring the grid sums the same terms in ascending order
    asc = oracle.run(u0[::-1, ::-1], 3, dim=2, shape=oracle.STAR, r=1, weights=w[::-1],
                     arith=oracle.ARITH_FMA)[::-1, ::-1]
    assert not np.array_equal(a, asc)
    assert np.max(np.abs(a - asc)) < 1e-14


def _fourier_lambda(offs, w, theta):
    return sum(wi * np.exp(1j * np.dot(theta, o)) for wi, o in zip(w, offs))


@pytest.mark.parametrize("dim,shape,ext,T", [
    (1, "star", (64,), 50), (2, "star", (16, 24), 20), (2, "box", (12, 20), 12), (3, "star", (8, 10, 12), 6)])
@pytest.mark.parametrize("arith", [oracle.ARITH_FMA, oracle.ARITH_UNFUSED])
def test_p2_fourier_periodic_jacobi(dim, shape, ext, T, arith):
    offs = exact.canonical_offsets(dim, shape, 1)
    w = inputs.normalized_weights(300 + dim, len(offs))      # non-symmetric: lambda is complex
    k = [1, 2, 3][:dim]
    theta = np.array([2 * np.pi * kk / n for kk, n in zip(k, ext)])
    idx = np.indices(ext)
    phase = sum(theta[d] * idx[d] for d in range(dim))
    u0 = np.cos(phase)
    lam = _fourier_lambda(offs, w, theta)
    expect = np.real(lam ** T * np.exp(1j * phase))
    got = oracle.run(u0, T, dim=dim, shape=SHAPES[shape], r=1, weights=w, bc=oracle.BC_PERIODIC, arith=arith)
    tol = (T * len(offs) + 10) * EPS * 4
    assert np.max(np.abs(got - expect)) < tol
    # a mirrored stencil (conjugate lambda) is far away, so a sign error would fail
    assert np.max(np.abs(np.real(np.conj(lam) ** T * np.exp(1j * phase)) - expect)) > 1e3 * tol


@pytest.mark.parametrize("N,kmode,a,b,T", [(31, 1, 0.5, 0.25, 100), (40, 3, 0.6, 0.2, 40)])
def test_p3_dirichlet_sine_mode(N, kmode, a, b, T):
    x = np.arange(1, N + 1)
    u0 = np.sin(kmode * np.pi * x / (N + 1))
    lam = a + 2 * b * np.cos(kmode * np.pi / (N + 1))
    got = oracle.run(u0, T, dim=1, shape=oracle.STAR, r=1, weights=[b, a, b])
    assert np.max(np.abs(got - lam ** T * u0)) < (3 * T + 10) * EPS * 4


def test_p3_dirichlet_sine_mode_2d():
    n0, n1, T = 14, 19, 30
    i, j = np.indices((n0, n1)) + 1
    u0 = np.sin(2 * np.pi * i / (n0 + 1)) * np.sin(np.pi * j / (n1 + 1))
    b0, b1, a = 0.15, 0.1, 0.5
    w = [b0, b1, a, b1, b0]                               # canonical: (-1,0),(0,-1),(0,0),(0,1),(1,0)
    lam = a + 2 * b0 * np.cos(2 * np.pi / (n0 + 1)) + 2 * b1 * np.cos(np.pi / (n1 + 1))
    got = oracle.run(u0, T, dim=2, shape=oracle.STAR, r=1, weights=w)
    assert np.max(np.abs(got - lam ** T * u0)) < (5 * T + 10) * EPS * 4


@pytest.mark.parametrize("dim,shape", [(1, "star"), (2, "star"), (2, "box"), (3, "star"), (3, "box")])
@pytest.mark.parametrize("method", ["jacobi", "gs"])
@pytest.mark.parametrize("bc", ["constant", "periodic"])
def test_p4_constant_field(dim, shape, method, bc):
    offs = exact.canonical_offsets(dim, shape, 1)
    k = len(offs)
    w = np.full(k, 1.0 / 32.0)
    w[k // 2] = 1.0 - (k - 1) / 32.0                      # dyadic, sums to exactly 1
    ext = (7, 6, 5)[:dim]
    c = 0.8125
    u0 = np.full(ext, c)
    got = oracle.run(u0, 9, dim=dim, shape=SHAPES[shape], r=1, weights=w, method=METHODS[method], bc=BCS[bc], c=c)
    assert np.all(got == c)
    # random normalised weights: within the rounding bound
    wr = inputs.normalized_weights(17, k)
    got = oracle.run(u0, 9, dim=dim, shape=SHAPES[shape], r=1, weights=wr, method=METHODS[method], bc=BCS[bc], c=c)
    assert np.max(np.abs(got - c)) < 9 * (2 * k + 2) * EPS


def test_p5_identity_and_shifts():
    u0 = inputs.grid(3, (17,))
    offs = exact.canonical_offsets(1, "star", 1)          # (-1,), (0,), (1,)
    for method in (oracle.JACOBI, oracle.GAUSS_SEIDEL):
        got = oracle.run(u0, 5, dim=1, shape=oracle.STAR, r=1, weights=[0, 1, 0], method=method)
        assert np.array_equal(got, u0)
    # periodic Jacobi with weight 1 on offset -1: u'[x] = u[x-1], a circular shift right per step
    got = oracle.run(u0, 5, dim=1, shape=oracle.STAR, r=1, weights=[1, 0, 0], bc=oracle.BC_PERIODIC)
    assert np.array_equal(got, np.roll(u0, 5))
    # Gauss-Seidel with weight 1 on +1: reads the not-yet-updated right neighbour, shifts left, c enters
    got = oracle.run(u0, 3, dim=1, shape=oracle.STAR, r=1, weights=[0, 0, 1], method=oracle.GAUSS_SEIDEL, c=0.25)
    assert np.array_equal(got, np.concatenate([u0[3:], [0.25] * 3]))
    # Gauss-Seidel with weight 1 on -1 reads the newest left value: one sweep spreads the halo value
    got = oracle.run(u0, 1, dim=1, shape=oracle.STAR, r=1, weights=[1, 0, 0], method=oracle.GAUSS_SEIDEL, c=0.0)
    assert np.all(got == 0.0)
    # 2D: weight 1 on (0,-1) in periodic Jacobi shifts every row right
    u2 = inputs.grid(4, (5, 8))
    got = oracle.run(u2, 3, dim=2, shape=oracle.STAR, r=1, weights=[0, 1, 0, 0, 0], bc=oracle.BC_PERIODIC)
    assert np.array_equal(got, np.roll(u2, 3, axis=1))
    assert offs == [(-1,), (0,), (1,)]


@pytest.mark.parametrize("dim,shape", [(1, "star"), (2, "star"), (2, "box"), (3, "star")])
def test_p6_gs_equals_jacobi_without_newest_terms(dim, shape):
    offs = exact.canonical_offsets(dim, shape, 1)
    w = inputs.normalized_weights(55, len(offs))
    zero = [o < tuple([0] * dim) for o in offs]           # lexicographically negative offsets
    w = np.where(zero, 0.0, w)
    ext = (9, 8, 7)[:dim]
    u0 = inputs.grid(66, ext)
    a = oracle.run(u0, 4, dim=dim, shape=SHAPES[shape], r=1, weights=w, method=oracle.JACOBI, c=0.3)
    b = oracle.run(u0, 4, dim=dim, shape=SHAPES[shape], r=1, weights=w, method=oracle.GAUSS_SEIDEL, c=0.3)
    assert np.array_equal(a, b)
    w2 = inputs.normalized_weights(55, len(offs))
    b2 = oracle.run(u0, 4, dim=dim, shape=SHAPES[shape], r=1, weights=w2, method=oracle.GAUSS_SEIDEL, c=0.3)
    a2 = oracle.run(u0, 4, dim=dim, shape=SHAPES[shape], r=1, weights=w2, method=oracle.JACOBI, c=0.3)
    assert not np.array_equal(a2, b2)


@pytest.mark.parametrize("dim,N", [(1, 16), (2, 10)])
def test_p7_young_gauss_seidel_rate(dim, N):
    """Model problem: GS spectral radius is the square of Jacobi's, cos^2(pi/(N+1))."""
    if dim == 1:
        w, shape, ext = [0.5, 0.0, 0.5], oracle.STAR, (N,)
    else:
        w, shape, ext = [0.25, 0.25, 0.0, 0.25, 0.25], oracle.STAR, (N, N)
    u = inputs.grid(9, ext) + 0.5
    rho = math.cos(math.pi / (N + 1)) ** 2
    u = oracle.run(u, 300, dim=dim, shape=shape, r=1, weights=w, method=oracle.GAUSS_SEIDEL)
    n0 = np.linalg.norm(u)
    u = oracle.run(u, 1, dim=dim, shape=shape, r=1, weights=w, method=oracle.GAUSS_SEIDEL)
    ratio = np.linalg.norm(u) / n0
    assert abs(ratio - rho) < 1e-6
    # Jacobi's own rate is the unsquared cos(pi/(N+1)), far from the GS rate
    assert abs(math.cos(math.pi / (N + 1)) - rho) > 1e-2


def test_offsets_canonical_order_and_counts():
    for dim in (1, 2, 3):
        for r in (1, 2, 3, 4):
            for shape in ("star", "box"):
                got = oracle.offsets(dim, SHAPES[shape], r)
                assert got == exact.canonical_offsets(dim, shape, r)
                assert len(got) == ((2 * dim * r + 1) if shape == "star" else (2 * r + 1) ** dim)
                assert got == sorted(got)


def test_rejects_bad_arguments():
    u = np.zeros(4)
    with pytest.raises(ValueError):
        oracle.run(u, 1, dim=1, shape=oracle.STAR, r=1, weights=[1, 2])            # K mismatch
    with pytest.raises(ValueError):
        oracle.run(u, 1, dim=1, shape=oracle.STAR, r=2, weights=[1] * 5, bc=oracle.BC_PERIODIC)  # ext < 2r+1
    with pytest.raises(ValueError):
        oracle.run(u, -1, dim=1, shape=oracle.STAR, r=1, weights=[1, 1, 1])
    got = oracle.run(u + 0.5, 0, dim=1, shape=oracle.STAR, r=1, weights=[1, 1, 1])
    assert np.array_equal(got, u + 0.5)


# ---- variable coefficients (a per-point weight field) -------------------------------------------

@pytest.mark.parametrize("dim,shape,ext", [(1, "star", (11,)), (2, "star", (5, 6)), (2, "box", (4, 5)),
                                           (3, "star", (3, 4, 4))])
@pytest.mark.parametrize("method", ["jacobi", "gs"])
@pytest.mark.parametrize("bc", ["constant", "periodic"])
def test_pvar_field_rounding_emulated(dim, shape, ext, method, bc):
    """Per-point weights: every rounding reproduced by the independent Fraction implementation."""
    offs = exact.canonical_offsets(dim, shape, 1)
    k = len(offs)
    field = inputs.uniform(401 + dim, k * int(np.prod(ext))).reshape((k,) + ext) / k
    u0 = inputs.grid(402 + dim, ext)
    for rounding, arith in (("fma", oracle.ARITH_FMA), ("unfused", oracle.ARITH_UNFUSED)):
        ref = exact.to_array(exact.run(u0, 2, dim=dim, shape=shape, r=1, weights=[0.0] * k, method=method, bc=bc,
                                       c=0.2, rounding=rounding, field=field), ext)
        got = oracle.run(u0, 2, dim=dim, shape=SHAPES[shape], r=1, weights=[0.0] * k, method=METHODS[method],
                         bc=BCS[bc], c=0.2, arith=arith, field=field)
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("method", [oracle.JACOBI, oracle.GAUSS_SEIDEL])
def test_pvar_uniform_field_equals_constant_weights(method):
    """A field that repeats the constant weights at every point gives the constant-weight result bit for bit."""
    w = inputs.normalized_weights(77, 9)
    u0 = inputs.grid(78, (13, 17))
    field = np.broadcast_to(np.asarray(w).reshape(9, 1, 1), (9, 13, 17)).copy()
    a = oracle.run(u0, 5, dim=2, shape=oracle.BOX, r=1, weights=w, method=method, c=0.4)
    b = oracle.run(u0, 5, dim=2, shape=oracle.BOX, r=1, weights=[0.0] * 9, method=method, c=0.4, field=field)
    assert np.array_equal(a, b)


def test_pvar_field_is_really_per_point():
    """Changing the weight of one point changes that point's first update and nothing else at T = 1 (Jacobi)."""
    w = inputs.normalized_weights(79, 3)
    u0 = inputs.grid(80, (20,))
    field = np.broadcast_to(np.asarray(w).reshape(3, 1), (3, 20)).copy()
    base = oracle.run(u0, 1, dim=1, shape=oracle.STAR, r=1, weights=w, field=field)
    field[1, 7] *= 0.5
    changed = oracle.run(u0, 1, dim=1, shape=oracle.STAR, r=1, weights=w, field=field)
    diff = np.nonzero(base != changed)[0]
    assert list(diff) == [7]
