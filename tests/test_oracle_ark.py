"""Pins of the oracle's ARK predictors (Section II tableaux) and of RIDC built on them
(Section III-D, Theorem 2), without any GPU.

  * The tableaux satisfy every additive Runge-Kutta order condition up to their order, in
    exact rational arithmetic (bicoloured rooted trees: one condition per tree and colouring
    of its vertices by the stiff/non-stiff part), and fail at least one of the next order.
  * One ARK step on a Fourier mode of the periodic problem equals the closed-form stability
    function R(z_S, z_N) = 1 + (z_S b^S + z_N b^N)^T (I - z_S A^S - z_N A^N)^-1 1 applied to
    the mode (the operators are diagonal in the Fourier basis).
  * Theorem 2: with a p0-th order predictor and first-order IMEX correctors, level j
    converges at order p0 + j against the semi-discrete exact solution under dt halving.
  * The lagged pipeline reproduces sequential IDC bit for bit with an ARK predictor too, and
    its start-up waits follow from the wider stencils.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

import inputs
import oracle
from oracle.ark import ARK3, ARK4, TABLEAUX, ark_step, predictor_order
from oracle.ridc import quadrature_nodes


# ---------------------------------------------------------------- order conditions
def _trees(order):
    """Rooted trees with `order` vertices, each a sorted tuple of child subtrees."""
    if order == 1:
        return [()]
    out = set()

    def forests(rem, bound):
        if rem == 0:
            yield ()
            return
        for k in range(1, rem + 1):
            for t in _trees(k):
                key = (k, t)
                if bound is not None and key > bound:
                    continue
                for rest in forests(rem - k, key):
                    yield (t,) + rest
    for ch in forests(order - 1, None):
        out.add(tuple(sorted(ch)))
    return sorted(out)


def _size(t):
    return 1 + sum(_size(c) for c in t)


def _gamma(t):
    g = _size(t)
    for c in t:
        g *= _gamma(c)
    return g


def _colourings(t):
    for col in "SN":
        for chs in itertools.product(*[list(_colourings(c)) for c in t]):
            yield (col, chs)


def _failed_conditions(tab, q):
    """Bicoloured trees of order q whose elementary weight differs from 1/gamma."""
    s = tab.stages
    A = {"S": [[tab.a_s(i, j) for j in range(s)] for i in range(s)],
         "N": [[tab.a_n(i, j) for j in range(s)] for i in range(s)]}
    b = {"S": list(tab.bS), "N": list(tab.bN)}

    def inner(ct, i):
        col, chs = ct
        return sum(A[col][i][j] * _prod(chs, j) for j in range(s))

    def _prod(chs, j):
        r = Fraction(1)
        for c in chs:
            r *= inner(c, j)
        return r

    bad, total = [], 0
    for t in _trees(q):
        for col, chs in _colourings(t):
            total += 1
            phi = sum(b[col][i] * _prod(chs, i) for i in range(s))
            if phi != Fraction(1, _gamma(t)):
                bad.append((t, col, chs))
    return bad, total


def test_tree_enumeration_counts():
    # 1, 1, 2, 4, 9 rooted trees with 1..5 vertices (OEIS A000081)
    assert [len(_trees(q)) for q in range(1, 6)] == [1, 1, 2, 4, 9]


@pytest.mark.parametrize("tab", [ARK3, ARK4], ids=lambda t: t.name)
def test_tableau_structure(tab):
    s = tab.stages
    for i in range(s):
        assert sum(tab.a_s(i, j) for j in range(s)) == tab.c[i]
        assert sum(tab.a_n(i, j) for j in range(s)) == tab.c[i]
        assert all(tab.a_s(i, j) == 0 for j in range(i + 1, s))   # diagonally implicit
        assert all(tab.a_n(i, j) == 0 for j in range(i, s))       # explicit
    assert tab.a_s(0, 0) == 0                                     # first stage explicit
    # stiffly accurate: the last stage is the new solution
    assert [tab.a_s(s - 1, j) for j in range(s)] == list(tab.bS)
    assert [tab.a_n(s - 1, j) for j in range(s)] == list(tab.bN)
    assert tab.bN[s - 1] == 0


@pytest.mark.parametrize("tab", [ARK3, ARK4], ids=lambda t: t.name)
def test_order_conditions_exact(tab):
    for q in range(1, tab.order + 1):
        bad, total = _failed_conditions(tab, q)
        assert total == 2 ** q * len(_trees(q))
        assert not bad, (tab.name, q, bad[:3])
    bad, _ = _failed_conditions(tab, tab.order + 1)
    assert bad, f"{tab.name} would be of order {tab.order + 1}"


# ---------------------------------------------------------------- one step on a Fourier mode
def _stability(tab, zS, zN):
    s = tab.stages
    AS = np.array([[float(tab.a_s(i, j)) for j in range(s)] for i in range(s)])
    AN = np.array([[float(tab.a_n(i, j)) for j in range(s)] for i in range(s)])
    bS = np.array([float(x) for x in tab.bS])
    bN = np.array([float(x) for x in tab.bN])
    Y = np.linalg.solve(np.eye(s) - zS * AS - zN * AN, np.ones(s, dtype=complex))
    return 1.0 + (zS * bS + zN * bN) @ Y


@pytest.mark.parametrize("tab", [ARK3, ARK4], ids=lambda t: t.name)
@pytest.mark.parametrize("k", [1, 5, 13])
def test_ark_step_on_a_fourier_mode_is_the_stability_function(tab, k):
    n, a, nu, dt = 64, 0.8, 0.02, 1.0 / 40
    prob = oracle.AdvDiff1DPeriodic(n, a, nu)
    h = 1.0 / n
    x = np.arange(n) * h
    theta = 2 * np.pi * k * x + 0.3
    sigma = 4 * np.sin(np.pi * k * h) ** 2 / h ** 2     # D e^{i theta} = -nu sigma e^{i theta}
    omega = np.sin(2 * np.pi * k * h) / h                # f^N e^{i theta} = -i a omega e^{..}
    R = _stability(tab, dt * (-nu * sigma), dt * (-1j * a * omega))
    got = ark_step(prob, np.sin(theta), dt, tab)
    want = np.imag(R * np.exp(1j * theta))
    assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, np.max(np.abs(want)))


# ---------------------------------------------------------------- Theorem 2
def _semi_discrete_exact(w, t):
    n = w.n
    h = 1.0 / n
    x = np.arange(n) / n
    u = np.zeros(n)
    for kk, (A, ph) in enumerate(zip(w.meta["amp"], w.meta["phase"])):
        k = kk + 1
        sig = 4 * np.sin(np.pi * k * h) ** 2 / h ** 2
        om = np.sin(2 * np.pi * k * h) / h
        u += A * np.exp(-w.nu[0] * sig * t) * np.sin(2 * np.pi * k * x + ph - w.a * om * t)
    return u


@pytest.mark.parametrize("predictor", ["ark3", "ark4"])
def test_theorem2_orders_per_level(predictor):
    """Level j of RIDC with a p0-th order ARK predictor and j FBE correctors converges at
    order p0 + j (observed slopes approach it from above on this problem)."""
    p0 = predictor_order(predictor)
    P = 4
    errs = []
    for N in (128, 256, 512):
        w = inputs.adv_diff_1d(n=32, nsteps=N, dt=1.0 / N)
        lv = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, N, P, all_levels=True,
                                    predictor=predictor)
        ex = _semi_discrete_exact(w, 1.0)
        errs.append([np.linalg.norm(l - ex) / np.linalg.norm(ex) for l in lv])
    errs = np.array(errs)
    slopes = np.log2(errs[-2] / errs[-1])
    for j in range(P):
        assert slopes[j] >= p0 + j - 0.15, (j, slopes)
    assert errs[-1][-1] > 1e-13        # still above rounding, so the slopes mean something


@pytest.mark.parametrize("predictor", ["ark3", "ark4"])
def test_ark_alone_is_the_order_one_ridc(predictor):
    """order = 1 is the ARK method alone; its observed order is p0."""
    p0 = predictor_order(predictor)
    errs = []
    for N in (64, 128, 256):
        w = inputs.adv_diff_1d(n=32, nsteps=N, dt=1.0 / N)
        got = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, N, 1, predictor=predictor)
        ex = _semi_discrete_exact(w, 1.0)
        errs.append(np.linalg.norm(got - ex) / np.linalg.norm(ex))
    assert np.log2(errs[-2] / errs[-1]) >= p0 - 0.1


def test_quadrature_nodes_reading():
    assert [quadrature_nodes(j) for j in range(1, 5)] == [2, 3, 4, 5]          # Section III-C
    assert [quadrature_nodes(j, "ark4") for j in range(1, 4)] == [5, 6, 7]
    assert [quadrature_nodes(j, "ark3") for j in range(1, 4)] == [4, 5, 6]


# ---------------------------------------------------------------- lagged pipeline
def _problems():
    w1 = inputs.adv_diff_1d(n=32, nsteps=1, dt=1.0 / 64)
    w2 = inputs.burgers_1d(n=40, nsteps=1, T=0.001)
    w3 = inputs.gray_scott_2d(n=12, nsteps=1, width=0.4)
    w4 = inputs.adv_diff_2d(n=10, nsteps=1, kmax=2, nu=2e-3, dt=1.0 / 20)
    return [(oracle.from_workload(w), w) for w in (w1, w2, w3, w4)]


@pytest.mark.parametrize("predictor", ["ark3", "ark4"])
def test_lagged_equals_sequential_with_ark_predictor(predictor):
    for prob, w in _problems():
        for order in (1, 2, 3, 4):
            for nsteps in (0, 1, 3, 7):
                a = oracle.ridc_sequential(prob, w.u0, w.dt, nsteps, order, predictor=predictor)
                b = oracle.ridc_lagged(prob, w.u0, w.dt, nsteps, order, predictor=predictor)
                np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("predictor", ["fbe", "ark3", "ark4"])
def test_lagged_startup_waits(predictor):
    """Level j first computes in pipeline step 1 + j (p0 - 1) + j (j + 1) / 2: it needs level
    j-1 at index p0 + j - 1 (the last node of its start-up stencil). With p0 = 1 this is the
    paper's wait of j (j + 1) / 2 steps (Section III-E)."""
    p0 = predictor_order(predictor)
    w = inputs.adv_diff_1d(n=16, nsteps=1, dt=1.0 / 64)
    P, N = 4, 12
    _, sched = oracle.ridc_lagged(oracle.from_workload(w), w.u0, w.dt, N, P,
                                  with_schedule=True, predictor=predictor)
    for j in range(P):
        first = next(s for s, lv in enumerate(sched) if j in lv) + 1
        assert first == 1 + j * (p0 - 1) + j * (j + 1) // 2, (j, first)


def test_tableaux_registry():
    assert set(TABLEAUX) == {"ark3", "ark4"}
    assert predictor_order("fbe") == 1 and predictor_order("ark3") == 3 and predictor_order("ark4") == 4
