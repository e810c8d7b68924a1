"""The paper's own 1D problems on the CUDA path (Section IV): periodic advection-diffusion
with upwind advection (restarts included) and viscous Burgers with Dirichlet walls, plus
grids that are not multiples of the warp width. Parity with the FP64 oracle <= 1e-12.

The two full-length runs of the paper (Burgers: 2000 steps; advection-diffusion: 4000 steps
to T = 40) use a bar of 5e-12 against the FP64 oracle. There the oracle's own rounding is the
larger error: it takes the direct form of eq. (corr), which adds O(1) terms every step, and the
same algorithm in long double (tests/test_oracle_extended.py, solutions stored by
tests/golden/make_extended.py) puts it 1.2e-12 (Burgers) and 2.9e-12 (advection-diffusion)
away from the exact evaluation. The CUDA path is held to those stored solutions directly, at
1e-13 (it is 7e-16 and 2.9e-15 away)."""
LONG_RUN_BAR = 5e-12
EXTENDED_BAR = 1e-13
import os
import sys

import numpy as np
import pytest

import inputs
import oracle
from paper_1209_4297_gb300 import Integrator
from tests.gpu_util import need_cuda, rel_l2

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_extended  # noqa: E402

pytestmark = pytest.mark.gpu


def _gpu(w, order=None, splits=None, restart_every=None):
    need_cuda()
    with Integrator.from_workload(w, order=order, restart_every=restart_every) as it:
        it.set_initial(w.u0)
        for s in (splits or [w.nsteps]):
            it.advance(s)
        return it.solution(), [it.level(j)[0] for j in range(order or w.order)]


@pytest.mark.parametrize("n", [8, 33, 100, 999, 1000, 1024])
def test_burgers_grids_match_oracle(n):
    w = inputs.burgers_1d(n=n, nsteps=40, T=0.02)
    got, levels = _gpu(w)
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, 40, 4, all_levels=True)
    for j in range(4):
        assert rel_l2(levels[j], ref[j]) <= 1e-12, j
    assert rel_l2(got, ref[-1]) <= 1e-12


@pytest.mark.parametrize("order", [1, 2, 3, 5, 8, 9, 12])
def test_burgers_orders_match_oracle(order):
    # orders above 8 put two levels on some CTAs of the 8-CTA cluster
    w = inputs.burgers_1d(n=200, nsteps=37, T=0.037, order=order)
    got, _ = _gpu(w)
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, 37, order)
    assert rel_l2(got, ref) <= 1e-12


def test_burgers_paper_workload_matches_oracle():
    """The paper's run: 999 interior nodes, T = 1, 2000 steps (the moving layer forms)."""
    w = inputs.burgers_1d()
    got, _ = _gpu(w, splits=[700, 1300])
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, w.nsteps, w.order)
    assert rel_l2(got, ref) <= LONG_RUN_BAR
    assert rel_l2(got, make_extended.load("burgers_paper")) <= EXTENDED_BAR


@pytest.mark.parametrize("a", [-0.1, 0.25])
@pytest.mark.parametrize("n", [40, 1000])
def test_upwind_matches_oracle(a, n):
    w = inputs.adv_diff_upwind_1d(n=n, nsteps=60, T=0.6, a=a, restarts=0)
    got, levels = _gpu(w)
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, 60, 4, all_levels=True)
    for j in range(4):
        assert rel_l2(levels[j], ref[j]) <= 1e-12, j


def test_upwind_paper_workload_with_restarts_matches_oracle():
    """The paper's run: dx = 1/1000, T = 40, 4000 steps, 10 restart intervals."""
    w = inputs.adv_diff_upwind_1d()
    got, _ = _gpu(w, splits=[1234, 2766])
    ref = oracle.ridc_restarted(oracle.from_workload(w), w.u0, w.dt, w.nsteps, 4, w.restart_every)
    assert rel_l2(got, ref) <= LONG_RUN_BAR
    assert rel_l2(got, make_extended.load("upwind_paper")) <= EXTENDED_BAR


@pytest.mark.parametrize("nsteps", [400, 1000])
def test_burgers_shorter_paper_runs_hold_the_fp64_bar(nsteps):
    w = inputs.burgers_1d(nsteps=nsteps, T=nsteps / 2000)
    got, _ = _gpu(w)
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, nsteps, w.order)
    assert rel_l2(got, ref) <= 1e-12


@pytest.mark.parametrize("n", [40, 100, 250])
def test_central_periodic_ragged_grids_match_oracle(n):
    w = inputs.adv_diff_1d(n=n, nsteps=30, dt=1.0 / 512)
    got, _ = _gpu(w)
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, 30, 4)
    assert rel_l2(got, ref) <= 1e-12


def test_burgers_split_is_bitwise_identical():
    w = inputs.burgers_1d(n=300, nsteps=50, T=0.05)
    a, _ = _gpu(w)
    b, _ = _gpu(w, splits=[1, 2, 3, 44])
    np.testing.assert_array_equal(a, b)
