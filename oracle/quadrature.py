"""Lagrange quadrature weights of the RIDC corrector (Section III-C), in exact rationals.

The j-th corrector integrates level j-1's right-hand side f = f^S + f^N over one step
[t_n, t_{n+1}] with the interpolating polynomial through j+1 equispaced nodes:
  * n >= j-1: the nodes t_{n+1-j}, ..., t_{n+1} (a window ending at t_{n+1});
  * n <  j-1: the fixed start-up nodes t_0, ..., t_j.
The paper prints the weight index range as k = 0..j-1; the sum it feeds has j+1 terms
(k = 0..j), which is the range used here.

Both cases are one family: with the first node t_b (b = max(0, n+1-j)) and the step's
offset m = n - b inside the stencil, node i sits at s = i (s = (t - t_b) / dt) and

    w[j][m][i] = int_m^{m+1} prod_{l != i} (s - l) / (i - l) ds,    i = 0..j,

so the integral is dt * sum_i w[j][m][i] * f(t_{b+i}). The steady stencil is m = j-1;
the start-up stencils are m = 0..j-2. Uniform steps make the table independent of n.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache


def _poly_mul_linear(coef: list[Fraction], root: int) -> list[Fraction]:
    """Multiply the polynomial sum coef[q] s^q by (s - root)."""
    out = [Fraction(0)] * (len(coef) + 1)
    for q, c in enumerate(coef):
        out[q + 1] += c
        out[q] -= c * root
    return out


@lru_cache(maxsize=None)
def lagrange_weights(j: int, m: int) -> tuple[Fraction, ...]:
    """Exact weights w[j][m][0..j] (node i at s = i, integral over s in [m, m+1])."""
    if j < 1 or not (0 <= m <= j - 1):
        raise ValueError(f"need j >= 1 and 0 <= m <= j-1, got j={j}, m={m}")
    out = []
    for i in range(j + 1):
        coef = [Fraction(1)]
        denom = Fraction(1)
        for l in range(j + 1):
            if l == i:
                continue
            coef = _poly_mul_linear(coef, l)
            denom *= (i - l)
        integral = sum(c * (Fraction(m + 1) ** (q + 1) - Fraction(m) ** (q + 1)) / (q + 1)
                       for q, c in enumerate(coef))
        out.append(integral / denom)
    return tuple(out)


def weight_table(order: int) -> list[list[list[float]]]:
    """w[j][m][i] as float64 for j = 1..order-1 (w[0] is empty: the predictor has none)."""
    table: list[list[list[float]]] = [[]]
    for j in range(1, order):
        table.append([[float(w) for w in lagrange_weights(j, m)] for m in range(j)])
    return table


def stencil(j: int, n: int) -> tuple[int, int]:
    """(b, m): first node index b and interval offset m of corrector j's step n -> n+1."""
    b = max(0, n + 1 - j)
    return b, n - b


def stencil_nodes(K: int, n: int) -> tuple[int, int]:
    """(b, m) of a K-node stencil for the step n -> n+1: the window t_b..t_{b+K-1} ends at
    t_{n+1} once n >= K-2, and is the fixed start-up window t_0..t_{K-1} before that. The
    weights are those of `lagrange_weights(K - 1, m)`. stencil(j, n) is the case K = j + 1."""
    b = max(0, n + 2 - K)
    return b, n - b
