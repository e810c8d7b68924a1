"""RIDC with an ARK predictor on the CUDA path (Section II tableaux, Section III-D Theorem 2),
through the C ABI, against the oracle.

Level 0 takes the paper's third- or fourth-order IMEX additive Runge-Kutta step (every
implicit stage one batched solve with (I - a_ii dt D)), the correctors stay first-order IMEX
with p0 + j quadrature nodes. Bars as for RIDC-FBE: FP64 path <= 1e-12 relative L2 against
the oracle; mixed path <= 1e-8 (the contract) and near the FP64 path (regression bar).
"""
import numpy as np
import pytest

import inputs
import oracle
from paper_1209_4297_gb300 import Integrator, RidcError
from tests.gpu_util import need_cuda, rel_l2

pytestmark = pytest.mark.gpu

RIDC_ERR_UNSUPPORTED = -6


def _gpu(w, predictor, order, precision="fp64", n_refine=2, splits=None, restart_every=None):
    need_cuda()
    with Integrator.from_workload(w, precision=precision, n_refine=n_refine, order=order,
                                  predictor=predictor, restart_every=restart_every) as it:
        it.set_initial(w.u0)
        for s in (splits or [w.nsteps]):
            it.advance(s)
        return it.solution(), [it.level(j)[0] for j in range(order)], it.progress()


def _oracle(w, predictor, order, nsteps=None, all_levels=False):
    return oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt,
                                  w.nsteps if nsteps is None else nsteps, order,
                                  all_levels=all_levels, predictor=predictor)


@pytest.mark.parametrize("predictor", ["ark3", "ark4"])
@pytest.mark.parametrize("order", [1, 2, 4])
@pytest.mark.parametrize("n", [32, 25])     # 25: odd n, the plain (unsplit) FP64 products
def test_gray_scott_fp64_every_level(predictor, order, n):
    w = inputs.gray_scott_2d(n=n, nsteps=22, width=0.3, seed=4)
    _, levels, prog = _gpu(w, predictor, order)
    ref = _oracle(w, predictor, order, all_levels=True)
    assert prog[-1] == 22
    for j in range(order):
        assert rel_l2(levels[j], ref[j]) <= 1e-12, (j, rel_l2(levels[j], ref[j]))


@pytest.mark.parametrize("predictor", ["ark3", "ark4"])
@pytest.mark.parametrize("n", [24, 21])     # 21: one species with n^2 odd (scalar loads)
def test_dirichlet_fp64(predictor, n):
    w = inputs.adv_diff_2d(n=n, nsteps=25, kmax=4, dt=1.0 / (2 * n), nu=2e-3)
    got, _, _ = _gpu(w, predictor, 3)
    assert rel_l2(got, _oracle(w, predictor, 3)) <= 1e-12


@pytest.mark.parametrize("predictor", ["ark3", "ark4"])
def test_short_runs_shorter_than_the_startup_stencil(predictor):
    """Runs of 0-3 steps: the lower levels run on to the top level's start-up nodes."""
    w = inputs.gray_scott_2d(n=16, nsteps=1, width=0.4, seed=1)
    for nsteps in (0, 1, 2, 3):
        w.nsteps = nsteps
        got, _, prog = _gpu(w, predictor, 4)
        assert prog[-1] == nsteps
        assert rel_l2(got, _oracle(w, predictor, 4)) <= 1e-12


@pytest.mark.parametrize("predictor,order", [("ark4", 8), ("ark3", 10)])
def test_widest_stencils(predictor, order):
    """p0 + order - 1 = 11 and 12: the widest quadrature stencils the library accepts."""
    w = inputs.gray_scott_2d(n=16, nsteps=40, width=0.4, seed=2)
    got, _, _ = _gpu(w, predictor, order)
    assert rel_l2(got, _oracle(w, predictor, order)) <= 5e-12


def test_split_advance_is_bitwise_identical():
    w = inputs.gray_scott_2d(n=32, nsteps=20, width=0.3)
    a, _, _ = _gpu(w, "ark4", 4)
    b, _, _ = _gpu(w, "ark4", 4, splits=[1, 4, 6, 9])
    np.testing.assert_array_equal(a, b)


def test_restarts_with_ark_predictor():
    w = inputs.gray_scott_2d(n=24, nsteps=30, width=0.3, seed=6)
    got, _, _ = _gpu(w, "ark3", 3, restart_every=8, splits=[5, 25])
    ref = oracle.ridc_restarted(oracle.from_workload(w), w.u0, w.dt, 30, 3, 8, predictor="ark3")
    assert rel_l2(got, ref) <= 1e-12


def test_checkpoint_resume_with_ark_predictor():
    need_cuda()
    w = inputs.gray_scott_2d(n=32, nsteps=18, width=0.3)
    kw = dict(order=4, predictor="ark4")
    with Integrator.from_workload(w, **kw) as it:
        it.set_initial(w.u0)
        it.advance(7)
        state = it.save_state()
        it.advance(11)
        want = it.solution()
    with Integrator.from_workload(w, **kw) as it2:
        it2.load_state(state)
        it2.advance(11)
        np.testing.assert_array_equal(it2.solution(), want)
    with Integrator.from_workload(w, order=4) as it3:      # another predictor: refused
        with pytest.raises(RidcError):
            it3.load_state(state)


# ---------------------------------------------------------------- mixed precision
@pytest.mark.parametrize("predictor", ["ark3", "ark4"])
def test_gray_scott_mixed_256_through_startup(predictor):
    """Mixed BF16x3 with two refinements; every ARK stage solve runs on the tensor cores with
    its own operator (I - a_ii dt D). 24 steps pass the start-up (level 3 of RIDC with ARK4
    starts in pipeline step 16)."""
    w = inputs.gray_scott_2d(n=256, nsteps=24, width=0.3, seed=2)
    got, levels, _ = _gpu(w, predictor, 4, precision="mixed_bf16x3")
    fp64, _, _ = _gpu(w, predictor, 4)
    ref = _oracle(w, predictor, 4, all_levels=True)
    for j in range(4):
        assert rel_l2(levels[j], ref[j]) <= 1e-8, j
    print(f"{predictor} mixed 256: vs oracle {rel_l2(got, ref[-1]):.3e}, "
          f"vs FP64 GPU {rel_l2(got, fp64):.3e}")
    assert rel_l2(got, ref[-1]) <= 1e-12
    assert rel_l2(got, fp64) <= 1e-13


def test_dirichlet_fp16_mixed_ark3():
    w = inputs.adv_diff_2d(n=256, nsteps=16, kmax=8, nu=1e-3)
    got, _, _ = _gpu(w, "ark3", 3, precision="mixed_fp16x3")
    fp64, _, _ = _gpu(w, "ark3", 3)
    assert rel_l2(got, _oracle(w, "ark3", 3)) <= 1e-8
    assert rel_l2(got, fp64) <= 1e-12


def test_gray_scott_2048_mixed_ark4_full_size_truncated():
    """The benchmark's grid with the ARK4 predictor, through start-up (order 7)."""
    w = inputs.gray_scott_2d(n=2048, nsteps=20)
    got, _, _ = _gpu(w, "ark4", 4, precision="mixed_bf16x3")
    assert rel_l2(got, _oracle(w, "ark4", 4)) <= 1e-8
    assert rel_l2(got, _oracle(w, "ark4", 4)) <= 1e-12


# ---------------------------------------------------------------- order on the GPU
def test_theorem2_order_on_the_gpu():
    """ARK4 predictor + one FBE corrector (order 5) on smooth Dirichlet data under dt halving,
    against a fine-step reference run on the same path."""
    need_cuda()
    n = 64
    base = inputs.adv_diff_2d(n=n, nsteps=1, kmax=4, nu=2e-3, a=0.5, b=-0.3)

    def run(nsteps):
        w = inputs.adv_diff_2d(n=n, nsteps=nsteps, kmax=4, nu=2e-3, a=0.5, b=-0.3,
                               dt=0.25 / nsteps)
        got, _, _ = _gpu(w, "ark4", 2)
        return got

    ref = run(512)
    errs = [rel_l2(run(N), ref) for N in (16, 32, 64)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert base.u0.shape == ref.shape
    assert slopes[-1] >= 4.7, (errs, slopes)


# ---------------------------------------------------------------- refusals
def test_unsupported_requests():
    need_cuda()
    w = inputs.gray_scott_2d(n=16, nsteps=1)
    with pytest.raises(RidcError) as e:      # 4 + 10 - 1 = 13 nodes: wider than 12
        Integrator.from_workload(w, order=10, predictor="ark4")
    assert e.value.code == RIDC_ERR_UNSUPPORTED
    w1 = inputs.adv_diff_1d(n=64, nsteps=1)
    with pytest.raises(RidcError):                   # 1D: the same width limit
        Integrator.from_workload(w1, order=11, predictor="ark3").close()


# ---------------------------------------------------------------- 1D (one SM per level)
@pytest.mark.parametrize("predictor", ["ark3", "ark4"])
def test_1d_periodic_workload_every_level(predictor):
    """The 1D periodic advection-diffusion workload (N = 256, dt = 1/512) with an ARK
    predictor and three correctors: order 6 (ARK3) or 7 (ARK4)."""
    w = inputs.adv_diff_1d(nsteps=96)
    _, levels, prog = _gpu(w, predictor, 4)
    ref = _oracle(w, predictor, 4, all_levels=True)
    assert prog == [96] * 4
    for j in range(4):
        assert rel_l2(levels[j], ref[j]) <= 1e-12, (j, rel_l2(levels[j], ref[j]))


@pytest.mark.parametrize("predictor,order", [("ark3", 1), ("ark4", 2), ("ark3", 6), ("ark4", 9)])
def test_1d_burgers_orders(predictor, order):
    """Burgers' Dirichlet walls (Sherman-Morrison with each stage's own operator); order 9
    with ARK4 puts two levels on CTA 0 of the 8-CTA cluster and the widest stencil (12)."""
    w = inputs.burgers_1d(n=200, nsteps=37, T=0.037, order=order)
    got, _, _ = _gpu(w, predictor, order)
    assert rel_l2(got, _oracle(w, predictor, order)) <= 1e-12


def test_1d_upwind_with_restarts_and_split_advance():
    w = inputs.adv_diff_upwind_1d(n=300, nsteps=60, T=0.6, restarts=0)
    a, _, _ = _gpu(w, "ark4", 3, restart_every=20)
    b, _, _ = _gpu(w, "ark4", 3, restart_every=20, splits=[7, 13, 40])
    np.testing.assert_array_equal(a, b)
    ref = oracle.ridc_restarted(oracle.from_workload(w), w.u0, w.dt, 60, 3, 20, predictor="ark4")
    assert rel_l2(a, ref) <= 1e-12


def test_theorem2_order_6_on_the_1d_workload():
    """ARK3 predictor + three first-order correctors on the 1D periodic workload's problem:
    observed order 3 + 3 = 6 against its semi-discrete exact solution, on the GPU."""
    def exact(w, t):
        n, h = w.n, 1.0 / w.n
        x = np.arange(n) / n
        u = np.zeros(n)
        for kk, (A, ph) in enumerate(zip(w.meta["amp"], w.meta["phase"])):
            k = kk + 1
            sig = 4 * np.sin(np.pi * k * h) ** 2 / h ** 2
            om = np.sin(2 * np.pi * k * h) / h
            u += A * np.exp(-w.nu[0] * sig * t) * np.sin(2 * np.pi * k * x + ph - w.a * om * t)
        return u

    errs = []
    for N in (128, 256, 512):
        w = inputs.adv_diff_1d(n=32, nsteps=N, dt=1.0 / N)
        got, _, _ = _gpu(w, "ark3", 4)
        errs.append(rel_l2(got, exact(w, 1.0)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert slopes[-1] >= 5.85, (errs, slopes)
