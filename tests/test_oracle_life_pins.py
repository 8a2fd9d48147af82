"""Pins of the Game of Life oracle (Section 3.4, "Game of life") against facts it does not compute itself.

- an independent brute-force restatement (numpy shifts of the whole grid) on tiny random grids;
- Conway's textbook patterns under B3S23 (block, beehive, blinker, glider, a glider around a torus);
- the B2S23 example worked by hand: a domino becomes two dominoes above and below it;
- rule-mask special cases (all die, all live, identity);
- symmetry: the rule is isotropic, so rotating or reflecting the input rotates or reflects the output,
  and on a torus translation commutes with a step (a dropped, doubled or misplaced neighbour fails);
- mutants of the C oracle, each caught by the pins above.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle.integer as L
from paper_2010_04868_gb300 import inputs


def brute(cells, T, bc, rule):
    """Whole-grid restatement: sum the 8 shifted copies of the grid, then look up the rule."""
    birth, survive = rule
    a = np.asarray(cells, dtype=np.int64)
    for _ in range(T):
        if bc == L.BC_PERIODIC:
            n = sum(np.roll(np.roll(a, di, 0), dj, 1) for di in (-1, 0, 1) for dj in (-1, 0, 1) if (di, dj) != (0, 0))
        else:
            p = np.pad(a, 1)
            n = sum(p[1 + di:1 + di + a.shape[0], 1 + dj:1 + dj + a.shape[1]]
                    for di in (-1, 0, 1) for dj in (-1, 0, 1) if (di, dj) != (0, 0))
        a = np.where(a == 1, (survive >> n) & 1, (birth >> n) & 1)
    return a.astype(np.uint8)


RULES = [L.B2S23, L.B3S23, (0b000001000, 0b000000110), (0b101010101, 0b010101010)]


@pytest.mark.parametrize("ext", [(1, 1), (1, 7), (7, 1), (3, 3), (5, 8), (9, 13)])
@pytest.mark.parametrize("bc", [L.BC_CONSTANT, L.BC_PERIODIC])
@pytest.mark.parametrize("rule", RULES)
def test_life_equals_brute_force(ext, bc, rule):
    if bc == L.BC_PERIODIC and min(ext) < 3:
        pytest.skip("the library requires periodic extents >= 3")
    for seed in range(3):
        c0 = inputs.cells(900 + seed, ext, 0.4)
        for T in (0, 1, 2, 7):
            assert np.array_equal(L.life(c0, T, bc=bc, rule=rule), brute(c0, T, bc, rule)), (seed, T)


def _place(n0, n1, pattern, i0, j0):
    g = np.zeros((n0, n1), np.uint8)
    p = np.array(pattern, np.uint8)
    g[i0:i0 + p.shape[0], j0:j0 + p.shape[1]] = p
    return g


def test_conway_still_lifes_and_oscillator():
    block = _place(6, 6, [[1, 1], [1, 1]], 2, 2)
    beehive = _place(7, 8, [[0, 1, 1, 0], [1, 0, 0, 1], [0, 1, 1, 0]], 2, 2)
    for g in (block, beehive):
        for T in (1, 5):
            assert np.array_equal(L.life(g, T, rule=L.B3S23), g)
    blinker_h = _place(5, 5, [[1, 1, 1]], 2, 1)
    blinker_v = _place(5, 5, [[1], [1], [1]], 1, 2)
    assert np.array_equal(L.life(blinker_h, 1, rule=L.B3S23), blinker_v)
    assert np.array_equal(L.life(blinker_h, 2, rule=L.B3S23), blinker_h)


GLIDER = [[0, 1, 0], [0, 0, 1], [1, 1, 1]]   # moves one cell down and one right every 4 generations


def test_conway_glider_moves_diagonally():
    g = _place(12, 12, GLIDER, 1, 1)
    assert np.array_equal(L.life(g, 4, rule=L.B3S23), _place(12, 12, GLIDER, 2, 2))
    assert np.array_equal(L.life(g, 16, rule=L.B3S23), _place(12, 12, GLIDER, 5, 5))


def test_conway_glider_circles_a_torus():
    g = _place(8, 8, GLIDER, 0, 0)
    assert np.array_equal(L.life(g, 32, bc=L.BC_PERIODIC, rule=L.B3S23), g)   # 4 generations per cell, 8 cells
    assert not np.array_equal(L.life(g, 16, bc=L.BC_PERIODIC, rule=L.B3S23), g)


def test_b2s23_domino_by_hand():
    """B2S23 (Section 3.4): each cell of a domino has 1 live neighbour and dies; the four dead cells
    that touch both (directly above and below) have 2 and are born; every other cell has at most 1."""
    g = np.zeros((6, 6), np.uint8)
    g[2, 2] = g[2, 3] = 1
    want = np.zeros((6, 6), np.uint8)
    want[1, 2] = want[1, 3] = want[3, 2] = want[3, 3] = 1
    assert np.array_equal(L.life(g, 1), want)


def test_rule_mask_special_cases():
    c0 = inputs.cells(931, (9, 11), 0.5)
    for bc in (L.BC_CONSTANT, L.BC_PERIODIC):
        assert not L.life(c0, 1, bc=bc, rule=(0, 0)).any()
        assert L.life(c0, 1, bc=bc, rule=(0x1FF, 0x1FF)).all()
        assert np.array_equal(L.life(c0, 3, bc=bc, rule=(0, 0x1FF)), c0)


@pytest.mark.parametrize("bc", [L.BC_CONSTANT, L.BC_PERIODIC])
def test_isotropy(bc):
    c0 = inputs.cells(941, (10, 10), 0.45)
    out = L.life(c0, 3, bc=bc)
    for k in (1, 2, 3):
        assert np.array_equal(L.life(np.rot90(c0, k), 3, bc=bc), np.rot90(out, k))
    assert np.array_equal(L.life(c0.T, 3, bc=bc), out.T)
    assert np.array_equal(L.life(c0[::-1], 3, bc=bc), out[::-1])


def test_torus_translation():
    c0 = inputs.cells(951, (9, 12), 0.45)
    out = L.life(c0, 4, bc=L.BC_PERIODIC)
    for di, dj in ((1, 0), (0, 1), (3, -5)):
        assert np.array_equal(L.life(np.roll(c0, (di, dj), (0, 1)), 4, bc=L.BC_PERIODIC), np.roll(out, (di, dj), (0, 1)))


def test_thread_count_does_not_matter():
    c0 = inputs.cells(961, (64, 80), 0.4)
    assert np.array_equal(L.life(c0, 5, nthreads=1), L.life(c0, 5, nthreads=4))


# ---- mutants: planted mistakes in copies of int_oracle.c -------------------------------------

SRC = os.path.join(os.path.dirname(L.__file__), "int_oracle.c")
MUTANTS = {
    "counts_itself": [("if (di != 0 || dj != 0) n +=", "n +=")],
    "drops_a_corner": [("if (di != 0 || dj != 0) n +=", "if ((di != 0 || dj != 0) && !(di == 1 && dj == 1)) n +=")],
    "rule_masks_swapped": [("((alive ? survive : birth) >> n)", "((alive ? birth : survive) >> n)")],
    "in_place_update": [("b[i * n1 + j] = (uint8_t)", "a[i * n1 + j] = (uint8_t)")],
    "periodic_as_constant": [("if (bc == OI_BC_PERIODIC) {", "if (0) {")],
    "transposed_wrap": [("j = ((j % n1) + n1) % n1;", "j = ((j % n0) + n0) % n0;")],
    "one_step_too_many": [("for (int64_t t = 0; t < T; ++t) {", "for (int64_t t = 0; t <= T; ++t) {")],
}


def _quick_pins(lib):
    run = lambda c, T, **kw: L.life(c, T, lib=lib, **kw)
    for ext, bc in (((5, 8), L.BC_CONSTANT), ((5, 8), L.BC_PERIODIC), ((9, 13), L.BC_PERIODIC)):
        for rule in (L.B2S23, L.B3S23):
            c0 = inputs.cells(970, ext, 0.4)
            for T in (1, 2):
                assert np.array_equal(run(c0, T, bc=bc, rule=rule), brute(c0, T, bc, rule))
    g = _place(8, 8, GLIDER, 0, 0)
    assert np.array_equal(run(g, 32, bc=L.BC_PERIODIC, rule=L.B3S23), g)


def _variant(tmp_path, name, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert old in src, (name, old)
        src = src.replace(old, new)
    c = tmp_path / (name + ".c")
    c.write_text(src)
    so = tmp_path / (name + ".so")
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(c)])
    return L.load(str(so))


def test_unmutated_life_oracle_passes(tmp_path):
    _quick_pins(_variant(tmp_path, "original", []))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_life_mutant_is_caught(tmp_path, name):
    with pytest.raises(AssertionError):
        _quick_pins(_variant(tmp_path, name, MUTANTS[name]))
