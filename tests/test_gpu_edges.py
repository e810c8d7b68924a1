"""Edge cases of the CUDA path through the C ABI: empty advances, the smallest and largest
grids each path accepts (and the first ones it refuses), the degenerate orders, exact fixed
points, and non-finite data.
"""
import os
import sys

import numpy as np
import pytest

import inputs
import oracle
from paper_1209_4297_gb300 import Batch, Integrator, RidcError
from tests.gpu_util import need_cuda, rel_l2

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))

pytestmark = pytest.mark.gpu

RIDC_ERR_NONFINITE, RIDC_ERR_UNSUPPORTED = -4, -6


def _oracle(w, nsteps, order=None):
    return oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, nsteps, order or w.order)


# ---------------------------------------------------------------- empty advances
@pytest.mark.parametrize("case", ["1d", "2d_fp64", "2d_mixed", "2d_fp16"])
def test_advance_by_zero_changes_nothing(case):
    need_cuda()
    if case == "1d":
        w, prec = inputs.adv_diff_1d(nsteps=9), "fp64"
    elif case == "2d_fp64":
        w, prec = inputs.gray_scott_2d(n=32, nsteps=9, width=0.3), "fp64"
    else:
        w = inputs.gray_scott_2d(n=256, nsteps=9, width=0.3)
        prec = "mixed_bf16x3" if case == "2d_mixed" else "mixed_fp16x3"
    with Integrator.from_workload(w, precision=prec) as it:
        it.set_initial(w.u0)
        it.advance(0)
        np.testing.assert_array_equal(it.solution(), w.u0.reshape(it.shape))
        assert it.time() == 0.0 and it.progress() == [0] * w.order
        it.advance(5)
        before, prog, t = it.solution(), it.progress(), it.time()
        it.advance(0)
        np.testing.assert_array_equal(it.solution(), before)
        assert it.progress() == prog and it.time() == t
        it.advance(4)
        got = it.solution()
    with Integrator.from_workload(w, precision=prec) as it:
        it.set_initial(w.u0)
        it.advance(9)
        np.testing.assert_array_equal(got, it.solution())


def test_batch_advance_by_zero_changes_nothing():
    need_cuda()
    ws = inputs.ensemble(3, nsteps=4)
    with Batch(ws, n_refine=1) as b:
        b.set_initial([w.u0[0] for w in ws])
        b.advance(0)
        for i, w in enumerate(ws):
            np.testing.assert_array_equal(b.solution(i), w.u0[0])


# ---------------------------------------------------------------- smallest grids
@pytest.mark.parametrize("kind", ["neumann", "dirichlet"])
@pytest.mark.parametrize("n", [4, 5, 6])
def test_smallest_2d_fp64_grids(kind, n):
    if kind == "neumann":
        w = inputs.gray_scott_2d(n=n, nsteps=12, width=0.5)
    else:
        w = inputs.adv_diff_2d(n=n, nsteps=12, kmax=2, dt=1.0 / (4 * n), nu=2e-3)
    need_cuda()
    with Integrator.from_workload(w) as it:
        it.set_initial(w.u0)
        it.advance(12)
        got = it.solution()
    assert rel_l2(got, _oracle(w, 12)) <= 1e-12


def test_smallest_1d_grid():
    need_cuda()
    w = inputs.adv_diff_1d(n=8, nsteps=40)
    with Integrator.from_workload(w) as it:
        it.set_initial(w.u0)
        it.advance(40)
        got = it.solution()
    assert rel_l2(got, _oracle(w, 40)) <= 1e-12


def test_smallest_sizes_below_are_refused():
    need_cuda()
    with pytest.raises(RidcError):
        Integrator("gray_scott_2d_neumann", 3, [2e-5, 1e-5], 0.5, 4, F=0.04, k=0.06)
    with pytest.raises(RidcError):
        Integrator("adv_diff_1d_periodic", 7, [0.01], 1.0 / 512, 4, a=1.0)


# ---------------------------------------------------------------- largest grids
@pytest.mark.parametrize("n,order,nsteps", [(9216, 4, 10), (5551, 12, 70)])
def test_largest_1d_grids(n, order, nsteps):
    """The largest sides the 1D kernel's shared memory holds, (L + 1) n256 + L n + 1 <= 28000
    doubles with L levels per CTA: order 4 (one level per CTA) n = 9216; order 12 (two)
    n = 5551, a ragged row. dt = h/4 and nu = 4h make mu = nu dt / h^2 = 1. With the default
    coefficients mu is 600-1700, and the Laplacian's cancellation alone puts any FP64 run
    2e-12 (order 4) to 4e-10 (order 12) away from an 80-bit run of the same algorithm.
    Order 12 keeps a 5e-12 bar even at mu = 1: its start-up weights (sum |w| up to 30) put
    both the oracle and the CUDA path 2-3e-12 from an 80-bit run after 70 steps."""
    need_cuda()
    w = inputs.adv_diff_1d(n=n, nsteps=nsteps, dt=0.25 / n, nu=4.0 / n)
    with Integrator.from_workload(w, order=order) as it:
        it.set_initial(w.u0)
        it.advance(nsteps)
        got = it.solution()
    assert rel_l2(got, _oracle(w, nsteps, order)) <= (1e-12 if order <= 8 else 5e-12)


def test_order12_against_the_extended_precision_solution():
    """RIDC-12 at mu = 1 (n = 256, 70 steps): both the FP64 oracle and the CUDA path sit about
    2-3e-12 from the long-double evaluation of the same algorithm (stored by
    tests/golden/make_extended.py; the oracle's distance is bounded on the CPU by
    tests/test_oracle_extended.py), which is why order 12 is compared with the oracle at 5e-12."""
    need_cuda()
    import make_extended
    w, _ = make_extended.cases()["order12_n256"]
    with Integrator.from_workload(w, order=12) as it:
        it.set_initial(w.u0)
        it.advance(w.nsteps)
        got = it.solution()
    assert rel_l2(got, make_extended.load("order12_n256")) <= 3.5e-12
    assert rel_l2(got, _oracle(w, w.nsteps, 12)) <= 5e-12


@pytest.mark.parametrize("kind,n,order,prec", [
    ("adv_diff_1d_periodic", 9217, 4, "fp64"),        # needs one more row of 256
    ("adv_diff_1d_periodic", 5552, 12, "fp64"),
    ("adv_diff_2d_dirichlet", 4352, 4, "mixed_bf16x3"),   # mixed: at most 4096
    ("adv_diff_2d_dirichlet", 4352, 4, "mixed_fp16x3"),
    ("adv_diff_2d_dirichlet", 16385, 1, "fp64"),       # FP64: at most 16384
])
def test_first_sizes_above_the_limits_are_unsupported(kind, n, order, prec):
    need_cuda()
    with pytest.raises(RidcError) as e:
        Integrator(kind, n, [1e-3], 1e-3, order, a=1.0, b=1.0, precision=prec)
    assert e.value.code == RIDC_ERR_UNSUPPORTED


# ---------------------------------------------------------------- degenerate orders and data
@pytest.mark.parametrize("prec", ["fp64", "mixed_bf16x3", "mixed_fp16x3"])
def test_order_one_is_fbe_in_2d(prec):
    """P = 1 is the FBE predictor alone (Section II, eq. (imex_diffusion))."""
    need_cuda()
    w = inputs.adv_diff_2d(n=256, nsteps=10, kmax=8, nu=1e-3)
    with Integrator.from_workload(w, precision=prec, order=1) as it:
        it.set_initial(w.u0)
        it.advance(10)
        got = it.solution()
    bar = 1e-12 if prec == "fp64" else 1e-8
    assert rel_l2(got, _oracle(w, 10, 1)) <= bar


@pytest.mark.parametrize("prec", ["fp64", "mixed_bf16x3", "mixed_fp16x3"])
def test_gray_scott_homogeneous_state_is_exact(prec):
    """(u, v) = (1, 0) is a fixed point: reaction 0, Laplacian of a constant 0, so every
    right-hand side and increment is exactly 0 on every level and pass."""
    need_cuda()
    n = 256
    w = inputs.gray_scott_2d(n=n, nsteps=20)
    u0 = np.stack([np.ones((n, n)), np.zeros((n, n))])
    with Integrator.from_workload(w, precision=prec) as it:
        it.set_initial(u0)
        it.advance(20)
        for j in range(w.order):
            np.testing.assert_array_equal(it.level(j)[0], u0)


def test_zero_field_stays_zero():
    need_cuda()
    w = inputs.adv_diff_2d(n=256, nsteps=8, kmax=4)
    with Integrator.from_workload(w, precision="mixed_fp16x3") as it:
        it.set_initial(np.zeros_like(w.u0))
        it.advance(8)
        assert not np.any(it.solution())


def test_non_finite_data_is_reported():
    need_cuda()
    for w, prec in ((inputs.adv_diff_1d(nsteps=6), "fp64"),
                    (inputs.gray_scott_2d(n=256, nsteps=6, width=0.3), "mixed_bf16x3")):
        u0 = w.u0.copy()
        u0.reshape(-1)[17] = np.nan
        with Integrator.from_workload(w, precision=prec) as it:
            it.set_initial(u0)
            it.advance(6)
            with pytest.raises(RidcError) as e:
                it.solution()
            assert e.value.code == RIDC_ERR_NONFINITE
