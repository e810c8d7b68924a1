"""Pins of the oracle's quadrature weights (Section III-C) against closed forms and invariants."""
import os
from fractions import Fraction

import pytest

from oracle.quadrature import lagrange_weights, stencil, weight_table

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "quadrature_weights.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, den = line.split("/")
        f = lhs.split()
        j, m = int(f[0]), int(f[1])
        rows.append((j, m, [Fraction(int(v), int(den)) for v in f[2:]]))
    return rows


@pytest.mark.parametrize("j,m,expect", _golden())
def test_textbook_rules(j, m, expect):
    assert list(lagrange_weights(j, m)) == expect


@pytest.mark.parametrize("j", range(1, 12))
def test_rows_sum_to_one_and_integrate_degree_j_exactly(j):
    for m in range(j):
        w = lagrange_weights(j, m)
        assert sum(w) == 1
        # interpolatory on j+1 nodes: exact for s^q, q <= j, on [m, m+1]
        for q in range(j + 1):
            exact = (Fraction(m + 1) ** (q + 1) - Fraction(m) ** (q + 1)) / (q + 1)
            assert sum(wi * Fraction(i) ** q for i, wi in enumerate(w)) == exact
        # and not exact one degree higher (the rule really has j+1 nodes)
        q = j + 1
        exact = (Fraction(m + 1) ** (q + 1) - Fraction(m) ** (q + 1)) / (q + 1)
        assert sum(wi * Fraction(i) ** q for i, wi in enumerate(w)) != exact or j % 2 == 0


@pytest.mark.parametrize("j", range(1, 12))
def test_reflection_symmetry(j):
    # reversing time maps interval m onto j-1-m and node i onto j-i
    for m in range(j):
        assert lagrange_weights(j, m) == tuple(reversed(lagrange_weights(j, j - 1 - m)))


def test_stencil_nodes_follow_section_iii_c():
    for j in range(1, 8):
        for n in range(0, 20):
            b, m = stencil(j, n)
            nodes = list(range(b, b + j + 1))
            if n >= j - 1:
                assert nodes == list(range(n + 1 - j, n + 2))   # t_{n+1-k}, k = 0..j
            else:
                assert nodes == list(range(0, j + 1))           # t_0 .. t_j
            assert nodes[m] == n and nodes[m + 1] == n + 1      # integrates [t_n, t_{n+1}]


def test_float_table_shape_and_rounding():
    t = weight_table(4)
    assert t[0] == [] and [len(r) for r in t[1:]] == [1, 2, 3]
    assert t[3][2] == [1 / 24, -5 / 24, 19 / 24, 9 / 24]


def test_bad_indices_rejected():
    with pytest.raises(ValueError):
        lagrange_weights(0, 0)
    with pytest.raises(ValueError):
        lagrange_weights(3, 3)
