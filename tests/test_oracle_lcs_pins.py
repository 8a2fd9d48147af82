"""Pins of the LCS oracle (Section 3.4, "Longest common subsequence") against facts it does not compute itself.

- brute force: on tiny strings, the longest subsequence of A found in each prefix of B, by enumerating
  every subsequence of A;
- the textbook example ABCBDAB / BDCABA (length 4, Cormen et al., Introduction to Algorithms, Section 15.4);
- an independent bit-parallel restatement (the row-difference bit vector of Allison and Dix, 1986, and
  Hyyro, 2004: V' = (V + (V & M)) | (V & ~M) per character of A, lcs[na][j] = zeros among the first j
  bits), computed with Python integers;
- properties: symmetry, LCS(A, A) = |A|, disjoint alphabets give 0, a common last character adds 1,
  each row step is 0 or 1;
- mutants of the C oracle, each caught.
"""
import itertools
import os
import subprocess

import numpy as np
import pytest

import oracle.integer as OI
from paper_2010_04868_gb300 import inputs


def _is_subseq(s, t):
    it = iter(t)
    return all(c in it for c in s)


def brute_row(A, B):
    row = []
    for j in range(len(B) + 1):
        best = 0
        for mask in range(1 << len(A)):
            sub = [A[i] for i in range(len(A)) if mask >> i & 1]
            if len(sub) > best and _is_subseq(sub, B[:j]):
                best = len(sub)
        row.append(best)
    return np.array(row, np.int32)


def bitparallel_row(A, B):
    nb = len(B)
    full = (1 << nb) - 1
    M = {}
    for j, c in enumerate(B):
        M[c] = M.get(c, 0) | (1 << j)
    V = full
    for c in A:
        U = V & M.get(c, 0)
        V = ((V + U) | (V & ~U)) & full
    return np.array([sum(1 for k in range(j) if not (V >> k) & 1) for j in range(nb + 1)], np.int32)


def _seq(seed, n, sigma):
    return inputs.sequence(seed, n, sigma)


@pytest.mark.parametrize("sigma", [2, 3, 4])
def test_lcs_row_equals_brute_force(sigma):
    for seed in range(12):
        A = list(_seq(1300 + seed, 1 + seed % 8, sigma))
        B = list(_seq(1400 + seed, seed % 9, sigma))
        assert np.array_equal(OI.lcs(np.array(A, np.uint8), np.array(B, np.uint8)), brute_row(A, B)), seed


def test_lcs_textbook_example():
    row = OI.lcs(b"ABCBDAB", b"BDCABA")
    assert row[-1] == 4
    assert np.array_equal(row, brute_row(list(b"ABCBDAB"), list(b"BDCABA")))


@pytest.mark.parametrize("sigma", [2, 4, 20, 256])
def test_lcs_row_equals_bit_parallel_restatement(sigma):
    for seed, (na, nb) in enumerate([(0, 5), (5, 0), (1, 1), (37, 64), (64, 65), (130, 300), (300, 129)]):
        A = _seq(1500 + seed, na, sigma)
        B = _seq(1600 + seed, nb, sigma)
        assert np.array_equal(OI.lcs(A, B), bitparallel_row(list(A), list(B))), (na, nb)


def test_lcs_properties():
    A = _seq(1701, 150, 4)
    B = _seq(1702, 170, 4)
    ab, ba = OI.lcs(A, B), OI.lcs(B, A)
    assert ab[-1] == ba[-1]
    assert OI.lcs(A, A)[-1] == len(A)
    assert OI.lcs(A, B + np.uint8(10))[-1] == 0
    c = np.array([3], np.uint8)
    assert OI.lcs(np.concatenate([A, c]), np.concatenate([B, c]))[-1] == ab[-1] + 1
    assert set(np.diff(ab)) <= {0, 1} and ab[0] == 0
    assert OI.lcs(A[:0], B)[-1] == 0 and len(OI.lcs(A, B[:0])) == 1


# ---- mutants of the C oracle -----------------------------------------------------------------

SRC = os.path.join(os.path.dirname(OI.__file__), "int_oracle.c")
MUTANTS = {
    "diag_is_left": [("diag + 1 : (up > left", "left + 1 : (up > left")],
    "max_ignores_left": [("(up > left ? up : left)", "up")],
    "match_adds_nothing": [("? diag + 1 :", "? diag :")],
    "diag_not_advanced": [("            diag = up;\n", "")],
    "compares_shifted_b": [("A[x - 1] == B[y - 1]", "A[x - 1] == B[y < nb ? y : y - 1]")],
}


def _variant(tmp_path, name, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert old in src, (name, old)
        src = src.replace(old, new)
    c = tmp_path / (name + ".c")
    c.write_text(src)
    so = tmp_path / (name + ".so")
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(c)])
    return OI.load(str(so))


def _quick(lib):
    for seed in range(6):
        A = list(_seq(1800 + seed, 6, 3))
        B = list(_seq(1900 + seed, 7, 3))
        assert np.array_equal(OI.lcs(np.array(A, np.uint8), np.array(B, np.uint8), lib=lib), brute_row(A, B))
    assert OI.lcs(b"ABCBDAB", b"BDCABA", lib=lib)[-1] == 4


def test_unmutated_lcs_oracle_passes(tmp_path):
    _quick(_variant(tmp_path, "original", []))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_lcs_mutant_is_caught(tmp_path, name):
    with pytest.raises(AssertionError):
        _quick(_variant(tmp_path, name, MUTANTS[name]))
