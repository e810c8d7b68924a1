"""Pins of the oracle on 1D periodic advection-diffusion (Sections II, III; Theorem 1).

Central differences map every Fourier mode exp(2 pi i k x) onto itself:
  f^N: multiplies by -i a w_k,   w_k = sin(2 pi k h) / h,
  D:   multiplies by -nu s_k,    s_k = 4 sin^2(pi k h) / h^2,
so the semi-discrete system has the exact solution
  u_i(t) = sum_k A_k exp(-nu s_k t) sin(2 pi k x_i + phi_k - a w_k t),
and one FBE step multiplies a mode by g_k = (1 - i a dt w_k) / (1 + nu dt s_k).
"""
import numpy as np
import pytest

import inputs
from oracle import AdvDiff1DPeriodic, fbe, from_workload, ridc_restarted, ridc_sequential


def _modes(n):
    h = 1.0 / n
    k = np.arange(n)
    return 4.0 * np.sin(np.pi * k * h) ** 2 / h ** 2, np.sin(2 * np.pi * k * h) / h


def _exact(w, t):
    n = w.n
    x = np.arange(n) / n
    sig, om = _modes(n)
    u = np.zeros(n)
    for kk, k in enumerate(w.meta["modes"]):
        u += w.meta["amp"][kk] * np.exp(-w.nu[0] * sig[k] * t) * np.sin(
            2 * np.pi * k * x + w.meta["phase"][kk] - w.a * om[k] * t)
    return u


@pytest.mark.parametrize("k", [1, 5, 37, 128])
def test_operators_act_on_fourier_modes(k):
    n, a, nu = 256, 0.7, 0.02
    p = AdvDiff1DPeriodic(n, a, nu)
    x = np.arange(n) / n
    sig, om = _modes(n)
    c, s = np.cos(2 * np.pi * k * x), np.sin(2 * np.pi * k * x)
    # f^N(sin) = -a w_k cos,  D(sin) = -nu s_k sin
    np.testing.assert_allclose(p.fN(s), -a * om[k] * c, atol=1e-10 * (1 + a * abs(om[k])))
    np.testing.assert_allclose(p.D(s), -nu * sig[k] * s, atol=1e-9 * (1 + nu * sig[k]))


@pytest.mark.parametrize("k", [1, 8, 64, 100])
def test_fbe_amplification_closed_form(k):
    """P = 1 is the IMEX step of eq. (imex_diffusion): each mode is multiplied by g_k."""
    n, a, nu, dt, steps = 256, 1.0, 0.01, 1.0 / 512, 7
    p = AdvDiff1DPeriodic(n, a, nu)
    x = np.arange(n) / n
    sig, om = _modes(n)
    theta = 2 * np.pi * k * x + 0.3
    g = (1 - 1j * a * dt * om[k]) / (1 + nu * dt * sig[k])
    got = ridc_sequential(p, np.sin(theta), dt, steps, order=1)
    want = np.imag(g ** steps * np.exp(1j * theta))
    np.testing.assert_allclose(got, want, atol=1e-13)
    np.testing.assert_array_equal(got, fbe(p, np.sin(theta), dt, steps)[-1])


def test_observed_order_per_level_theorem_1():
    """Level j converges at order j+1 (each correction adds one order); RIDC4 at order 4."""
    w = inputs.adv_diff_1d()
    p = from_workload(w)
    ue = _exact(w, 1.0)
    errs = []
    for nt in (256, 512, 1024, 2048):
        levs = ridc_sequential(p, w.u0, 1.0 / nt, nt, 4, all_levels=True)
        errs.append([np.linalg.norm(l - ue) / np.linalg.norm(ue) for l in levs])
    errs = np.array(errs)
    slopes = np.log2(errs[-2] / errs[-1])
    for j in range(4):
        assert abs(slopes[j] - (j + 1)) < 0.25, (j, slopes)
    assert errs[-1, 3] < 2e-7


def test_small_run_shorter_than_startup_stencil():
    """nsteps < order-1: the lower levels run on to t_{order-1}; results stay finite and
    one step of RIDC4 differs from one FBE step only at the corrector level."""
    w = inputs.adv_diff_1d()
    p = from_workload(w)
    levs = ridc_sequential(p, w.u0, w.dt, 1, 4, all_levels=True)
    assert all(np.isfinite(l).all() for l in levs)
    np.testing.assert_array_equal(levs[0], fbe(p, w.u0, w.dt, 1)[1])


def test_zero_steps_is_identity():
    w = inputs.adv_diff_1d()
    p = from_workload(w)
    np.testing.assert_array_equal(ridc_sequential(p, w.u0, w.dt, 0, 4), w.u0)


# ---------------------------------------------------------------- restarts (Section III-E)
@pytest.mark.parametrize("every", [1, 3, 7, 20])
def test_restarted_fbe_is_fbe(every):
    """With one level the most corrected solution is the FBE state itself, so restarting
    from it at any interval must reproduce the plain FBE run bit for bit (this fails if a
    restart loses or repeats a step, or hands over the wrong state)."""
    w = inputs.adv_diff_1d(n=64, nsteps=20, dt=1.0 / 256)
    p = from_workload(w)
    plain = fbe(p, w.u0, w.dt, 20)[-1]
    np.testing.assert_array_equal(ridc_restarted(p, w.u0, w.dt, 20, 1, every), plain)


def test_restarted_without_restart_is_plain():
    w = inputs.adv_diff_1d(n=64, nsteps=12, dt=1.0 / 256)
    p = from_workload(w)
    plain = ridc_sequential(p, w.u0, w.dt, 12, 4)
    np.testing.assert_array_equal(ridc_restarted(p, w.u0, w.dt, 12, 4, 0), plain)
    np.testing.assert_array_equal(ridc_restarted(p, w.u0, w.dt, 12, 4, 12), plain)


def test_error_falls_as_restarts_increase():
    """Section IV-A (figure of RIDC4 error against restarts): on advection-diffusion to
    T = 40 with a fixed 4000 steps, the final error of RIDC4 falls as restarts are added.
    Here: u0 = 2 + sin(2 pi x), a = 0.1, nu = 1e-3, central differences on 128 points, error
    against the semi-discrete exact solution (time error only); 0, 1, 3 and 9 restarts."""
    n, a, nu, T, nt = 128, 0.1, 1e-3, 40.0, 4000
    p = AdvDiff1DPeriodic(n, a, nu)
    x = np.arange(n) / n
    sig, om = _modes(n)
    u0 = 2.0 + np.sin(2 * np.pi * x)
    exact = 2.0 + np.exp(-nu * sig[1] * T) * np.sin(2 * np.pi * x - a * om[1] * T)
    errs = []
    for restarts in (0, 1, 3, 9):
        u = ridc_restarted(p, u0, T / nt, nt, 4, nt // (restarts + 1))
        errs.append(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    assert all(e1 < 0.5 * e0 for e0, e1 in zip(errs, errs[1:])), errs


@pytest.mark.parametrize("order", [2, 4])
def test_restarts_fall_at_fixed_times(order):
    """Restarts happen at fixed multiples of the interval, so running to a restart time and
    continuing from there gives the same numbers as one run (this fails if a piece is
    longer or shorter than the interval)."""
    w = inputs.adv_diff_1d(n=64, nsteps=23, dt=1.0 / 256)
    p = from_workload(w)
    every = 5
    one = ridc_restarted(p, w.u0, w.dt, 2 * every + 3, order, every)
    mid = ridc_restarted(p, w.u0, w.dt, every, order, every)
    two = ridc_restarted(p, mid, w.dt, every + 3, order, every)
    np.testing.assert_array_equal(one, two)
