"""The identity behind the lagged pipeline (Section III-E): running the levels staggered, each
advancing as soon as the level below has produced its inputs, gives exactly the numbers of
classic sequential IDC. Pinned on the oracle with an independent pipelined driver, bit for
bit, together with the start-up the paper describes: level j first computes in pipeline step
j(j+1)/2 + 1 (it waits j(j+1)/2 steps), after which it advances in every step until it reaches
t_N, so a run of N_t steps takes N_t + P(P-1)/2 pipeline steps.
"""
import numpy as np
import pytest

import inputs
from oracle import (AdvDiff1DPeriodic, Burgers1DDirichlet, from_workload, ridc_lagged,
                    ridc_sequential)


def _problems():
    yield "adv_diff_1d", AdvDiff1DPeriodic(64, 1.0, 0.01), inputs.adv_diff_1d(n=64).u0, 1.0 / 256
    p = Burgers1DDirichlet(31, 1e-2)
    x = np.arange(1, 32) * p.h
    yield "burgers", p, np.sin(2 * np.pi * x) + 0.3 * np.sin(np.pi * x), 1.0 / 64
    w = inputs.gray_scott_2d(n=16, nsteps=1, width=0.3, seed=1)
    yield "gray_scott", from_workload(w), w.u0, w.dt
    w = inputs.adv_diff_2d(n=12, nsteps=1, kmax=3, nu=2e-3)
    yield "dirichlet_2d", from_workload(w), w.u0, w.dt


@pytest.mark.parametrize("case", list(range(4)))
@pytest.mark.parametrize("order", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("nsteps", [0, 1, 2, 5, 13])
def test_lagged_pipeline_equals_sequential_bit_for_bit(case, order, nsteps):
    name, prob, y0, dt = list(_problems())[case]
    lag = ridc_lagged(prob, y0, dt, nsteps, order)
    seq = ridc_sequential(prob, y0, dt, nsteps, order)
    assert np.array_equal(lag, seq), name


@pytest.mark.parametrize("order", [2, 3, 4, 5, 8])
def test_start_up_waits_follow_the_paper(order):
    prob = AdvDiff1DPeriodic(16, 1.0, 0.01)
    y0 = inputs.adv_diff_1d(n=16).u0
    nsteps = 3 * order
    _, sched = ridc_lagged(prob, y0, 1.0 / 128, nsteps, order, with_schedule=True)
    first = [next(s for s, lv in enumerate(sched) if j in lv) for j in range(order)]
    assert first == [j * (j + 1) // 2 for j in range(order)], first
    assert len(sched) == nsteps + order * (order - 1) // 2
    # once started, a level advances in every step until it reaches t_N; the lower levels
    # get there first and then idle while the upper ones drain (Section III-E)
    for j in range(order):
        steps = [s for s, lv in enumerate(sched) if j in lv]
        assert steps == list(range(first[j], first[j] + nsteps)), (j, steps)
