"""Additive Runge-Kutta (IMEX) predictors for RIDC (Section II tableaux; Section III-D, Theorem 2).

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; see the package docstring).

Section II couples an s-stage diagonally implicit RK method (A^S, b^S) for the stiff term
with an explicit one (A^N, b^N) for the non-stiff term, on shared abscissae c. One step from
y_n computes the stages

    Y_i = y_n + dt sum_{j<=i} a^S_ij K^S_j + dt sum_{j<i} a^N_ij K^N_j,
    K^S_i = f^S(Y_i),   K^N_i = f^N(Y_i),

and then y_{n+1} = y_n + dt sum_i (b^S_i K^S_i + b^N_i K^N_i). With the linear stiff part
f^S = D y of every problem here, the implicit stage is one linear solve:

    (I - dt a^S_ii D) Y_i = y_n + dt sum_{j<i} (a^S_ij K^S_j + a^N_ij K^N_j),

and a stage with a^S_ii = 0 is explicit. Theorem 2: RIDC whose predictor is a p0-th order ARK
method and whose correctors are first-order IMEX (FBE) steps has order p0 + (number of
correctors), provided the quadrature of each corrector is accurate enough; see
`oracle.ridc.quadrature_nodes` for the stencil reading.

The two tableaux are the paper's third- and fourth-order IMEX methods. The third-order one is
garbled in the printed source; the reading used (rows of A^S / A^N, stage by stage) is

    c    A^S                              A^N
    0    0                                .
    1/2  0    1/2                         1/2
    1/2  1/4 -5/12 2/3                    1/4 1/4
    1    2   -7/2  1/2  2                 0   1   0
    1    1/6  0    2/3 -5/6  1            1/6 0   2/3 1/6
    b^S = last row of A^S, b^N = (1/6, 0, 2/3, 1/6, 0)

which satisfies every additive-RK order condition up to order 3 exactly (and the row sums
equal c for both parts); the fourth-order tableau satisfies every condition up to order 4.
Both are checked in exact rational arithmetic by tests/test_oracle_ark.py.
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction


def _row(*vals) -> tuple[Fraction, ...]:
    return tuple(Fraction(v) for v in vals)


@dataclass(frozen=True)
class ArkTableau:
    """An IMEX additive RK method: A^S lower triangular (diagonally implicit), A^N strictly
    lower triangular (explicit), shared abscissae c, weights b^S and b^N; exact rationals."""
    name: str
    order: int
    c: tuple
    AS: tuple       # AS[i][j], j <= i
    AN: tuple       # AN[i][j], j < i
    bS: tuple
    bN: tuple

    @property
    def stages(self) -> int:
        return len(self.bS)

    def a_s(self, i: int, j: int) -> Fraction:
        row = self.AS[i]
        return row[j] if j < len(row) else Fraction(0)

    def a_n(self, i: int, j: int) -> Fraction:
        row = self.AN[i]
        return row[j] if j < len(row) else Fraction(0)


# Section II, third-order IMEX method (reading above)
ARK3 = ArkTableau(
    name="ark3", order=3,
    c=_row(0, "1/2", "1/2", 1, 1),
    AS=(_row(0),
        _row(0, "1/2"),
        _row("1/4", "-5/12", "2/3"),
        _row(2, "-7/2", "1/2", 2),
        _row("1/6", 0, "2/3", "-5/6", 1)),
    AN=(_row(),
        _row("1/2"),
        _row("1/4", "1/4"),
        _row(0, 1, 0),
        _row("1/6", 0, "2/3", "1/6")),
    bS=_row("1/6", 0, "2/3", "-5/6", 1),
    bN=_row("1/6", 0, "2/3", "1/6", 0),
)

# Section II, fourth-order IMEX method: the printed DIRK and explicit RK tableaux
ARK4 = ArkTableau(
    name="ark4", order=4,
    c=_row(0, "1/3", "1/3", "1/2", "1/2", 1, 1),
    AS=(_row(0),
        _row("-1/6", "1/2"),
        _row("1/6", "-1/3", "1/2"),
        _row("3/8", "-3/8", 0, "1/2"),
        _row("1/8", 0, "3/8", "-1/2", "1/2"),
        _row("-1/2", 0, 3, -3, 1, "1/2"),
        _row("1/6", 0, 0, 0, "2/3", "-1/2", "2/3")),
    AN=(_row(),
        _row("1/3"),
        _row("1/6", "1/6"),
        _row("1/8", 0, "3/8"),
        _row("1/8", 0, "3/8", 0),
        _row("1/2", 0, "-3/2", 0, 2),
        _row("1/6", 0, 0, 0, "2/3", "1/6")),
    bS=_row("1/6", 0, 0, 0, "2/3", "-1/2", "2/3"),
    bN=_row("1/6", 0, 0, 0, "2/3", "1/6", 0),
)

TABLEAUX = {"ark3": ARK3, "ark4": ARK4}


def predictor_order(predictor: str) -> int:
    """p0 of a predictor name: 'fbe' (Section II's first-order IMEX step) or an ARK tableau."""
    if predictor == "fbe":
        return 1
    return TABLEAUX[predictor].order


def ark_step(problem, y, dt: float, tab: ArkTableau):
    """One step of the IMEX additive RK method `tab` from y (Section II), with the stage
    equations solved as written: every implicit stage is one solve with (I - dt a^S_ii D)."""
    s = tab.stages
    KS, KN = [], []
    for i in range(s):
        rhs = y.copy()
        for j in range(i):
            if tab.a_s(i, j) != 0:
                rhs = rhs + dt * float(tab.a_s(i, j)) * KS[j]
            if tab.a_n(i, j) != 0:
                rhs = rhs + dt * float(tab.a_n(i, j)) * KN[j]
        aii = tab.a_s(i, i)
        Yi = problem.solve(rhs, dt * float(aii)) if aii != 0 else rhs
        KS.append(problem.D(Yi))
        KN.append(problem.fN(Yi))
    out = y.copy()
    for i in range(s):
        if tab.bS[i] != 0:
            out = out + dt * float(tab.bS[i]) * KS[i]
        if tab.bN[i] != 0:
            out = out + dt * float(tab.bN[i]) * KN[i]
    return out
