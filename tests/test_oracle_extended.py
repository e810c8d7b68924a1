"""The extended-precision oracle and the rounding level of the FP64 oracle on long runs.

The FP64 oracle evaluates eq. (corr) in its direct form, which adds O(1) terms every step, so
over the paper's long 1D runs its own rounding reaches the 1e-12 level. The same algorithm run
in long double (oracle.problems, dtype=np.longdouble) measures that rounding directly:

  * pins of the long-double machinery: its solve's residual is at the long-double rounding
    level, it agrees with the FP64 solve, and a short run agrees with the FP64 oracle;
  * the stored extended-precision solutions (tests/golden/extended_*.txt, written by
    tests/golden/make_extended.py, which calls only the oracle) are reproduced;
  * the FP64 oracle's distance from them on the paper's Burgers run (Section IV-B: 1.2e-12),
    its advection-diffusion run with restarts (Section IV-A: 2.9e-12) and a 70-step RIDC-12
    run (2.9e-12, order 12's start-up weights reach sum |w| = 30) is bounded.

Those bounds are why the GPU parity tests of these three runs use 5e-12 against the FP64
oracle; the GPU tests also hold the CUDA path to the stored extended-precision solutions.
"""
import os
import sys

import numpy as np
import pytest

import inputs
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_extended  # noqa: E402

LD = np.longdouble
EXTENDED = np.finfo(LD).eps < 1e-18
needs_extended = pytest.mark.skipif(not EXTENDED, reason="long double is FP64 on this machine")


def _rel(a, b):
    a = np.asarray(a, dtype=LD)
    b = np.asarray(b, dtype=LD)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@needs_extended
@pytest.mark.parametrize("kind", ["periodic", "upwind", "burgers"])
def test_extended_solve_residual_and_agreement(kind):
    n, dt = 200, 1.0 / 256
    if kind == "periodic":
        p64, pld = oracle.AdvDiff1DPeriodic(n, 1.0, 0.05), oracle.AdvDiff1DPeriodic(n, 1.0, 0.05, LD)
    elif kind == "upwind":
        p64, pld = (oracle.AdvDiff1DUpwindPeriodic(n, -0.3, 0.05),
                    oracle.AdvDiff1DUpwindPeriodic(n, -0.3, 0.05, LD))
    else:
        p64, pld = oracle.Burgers1DDirichlet(n, 0.05), oracle.Burgers1DDirichlet(n, 0.05, LD)
    r = np.random.default_rng(3).standard_normal(n)
    x = pld.solve(r.astype(LD), dt)
    assert x.dtype == LD
    res = r.astype(LD) - (x - dt * pld.D(x))             # (I - dt D) x = r, in long double
    assert float(np.linalg.norm(res) / np.linalg.norm(r.astype(LD))) <= 1e-17
    assert _rel(x, p64.solve(r, dt)) <= 1e-14
    # the explicit terms are the same functions, evaluated in long double
    assert _rel(pld.fN(x), p64.fN(x.astype(np.float64))) <= 1e-14


@needs_extended
def test_extended_short_run_agrees_with_fp64_oracle():
    w = inputs.burgers_1d(n=100, nsteps=30, T=0.03)
    a = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, 30, 4)
    b = oracle.ridc_sequential(oracle.from_workload(w, LD), w.u0, w.dt, 30, 4, dtype=LD)
    assert b.dtype == LD
    assert _rel(a, b) <= 1e-14


def test_extended_precision_is_1d_only():
    with pytest.raises(ValueError):
        oracle.from_workload(inputs.gray_scott_2d(n=8, nsteps=1), LD)


# FP64 oracle against the extended-precision solution: measured 1.22e-12, 2.89e-12, 2.86e-12
FP64_ORACLE_BOUND = {"burgers_paper": 1.5e-12, "upwind_paper": 3.5e-12, "order12_n256": 3.5e-12}


@needs_extended
@pytest.mark.parametrize("name", sorted(FP64_ORACLE_BOUND))
def test_stored_extended_solutions_and_fp64_oracle_rounding(name):
    w, run = make_extended.cases()[name]
    stored = make_extended.load(name)
    ext = run(oracle.from_workload(w, LD), LD)
    assert _rel(stored, ext) <= 1e-16                  # the file is this computation
    fp64 = run(oracle.from_workload(w), np.float64)
    err = _rel(fp64, stored)
    assert err <= FP64_ORACLE_BOUND[name], err
    assert err >= 1e-14                                 # the effect the bars account for is real
