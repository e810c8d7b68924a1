"""Pins of the oracle on the paper's own 1D problems (Section IV): periodic
advection-diffusion with upwind advection and viscous Burgers with Dirichlet walls.

Upwind differences are circulant, so every Fourier mode exp(2 pi i k x) is an eigenvector:
  f^N: multiplies by s_k = -a (1 - exp(-i phi)) / h   (a >= 0),
                      s_k = -a (exp(i phi) - 1) / h   (a < 0),     phi = 2 pi k h,
  D:   multiplies by -nu sigma_k, sigma_k = 4 sin^2(phi / 2) / h^2,
which gives the semi-discrete exact solution and the FBE amplification factor in closed
form. Burgers has none; its flux, walls and solver are pinned one by one.
"""
import numpy as np
import pytest
import scipy.fft
from scipy.integrate import solve_ivp

import inputs
from oracle import (AdvDiff1DUpwindPeriodic, Burgers1DDirichlet, from_workload, ridc_restarted,
                    ridc_sequential)


def _symbol(n, a, nu, k):
    h = 1.0 / n
    phi = 2 * np.pi * k * h
    s = -a * (1 - np.exp(-1j * phi)) / h if a >= 0 else -a * (np.exp(1j * phi) - 1) / h
    return s, 4.0 * np.sin(phi / 2) ** 2 / h ** 2


# ---------------------------------------------------------------- upwind advection-diffusion
@pytest.mark.parametrize("a", [-0.1, 0.3])
@pytest.mark.parametrize("k", [1, 7, 250])
def test_upwind_operator_on_fourier_modes(a, k):
    n, nu = 1000, 1e-3
    p = AdvDiff1DUpwindPeriodic(n, a, nu)
    x = np.arange(n) / n
    s, sig = _symbol(n, a, nu, k)
    mode = np.exp(2j * np.pi * k * x)
    got = p.fN(mode.real) + 1j * p.fN(mode.imag)
    np.testing.assert_allclose(got, s * mode, atol=1e-9 * (1 + abs(s)))
    got = p.D(mode.real) + 1j * p.D(mode.imag)
    np.testing.assert_allclose(got, -nu * sig * mode, atol=1e-9 * (1 + nu * sig))


@pytest.mark.parametrize("a", [-0.1, 0.3])
def test_upwind_fbe_amplification(a):
    n, nu, dt, steps, k = 1000, 1e-3, 0.01, 9, 3
    p = AdvDiff1DUpwindPeriodic(n, a, nu)
    x = np.arange(n) / n
    s, sig = _symbol(n, a, nu, k)
    g = (1 + dt * s) / (1 + nu * dt * sig)
    theta = 2 * np.pi * k * x + 0.4
    got = ridc_sequential(p, np.sin(theta), dt, steps, order=1)
    np.testing.assert_allclose(got, np.imag(g ** steps * np.exp(1j * theta)), atol=1e-13)


def test_upwind_paper_problem_is_fourth_order():
    """Theorem 1 on the paper's advection-diffusion problem (u0 = 2 + sin(2 pi x), dx = 1/1000,
    c = 0.1, d = 1e-3), shortened to T = 4: RIDC4 against the semi-discrete exact solution."""
    T = 4.0
    errs = []
    for nt in (50, 100, 200):
        w = inputs.adv_diff_upwind_1d(nsteps=nt, T=T, restarts=0)
        s, sig = _symbol(w.n, w.a, w.nu[0], 1)
        x = np.arange(w.n) / w.n
        exact = 2.0 + np.imag(np.exp((s - w.nu[0] * sig) * T) * np.exp(2j * np.pi * x))
        u = ridc_sequential(from_workload(w), w.u0, w.dt, nt, 4)
        errs.append(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 3.7), (errs, slopes)


def test_upwind_paper_workload_restarts_help():
    """The paper's run (T = 40, 4000 steps) with 10 restart intervals is more accurate than
    without restarts (Section IV-A)."""
    errs = {}
    for restarts in (0, 10):
        w = inputs.adv_diff_upwind_1d(restarts=restarts)
        s, sig = _symbol(w.n, w.a, w.nu[0], 1)
        x = np.arange(w.n) / w.n
        exact = 2.0 + np.imag(np.exp((s - w.nu[0] * sig) * 40.0) * np.exp(2j * np.pi * x))
        u = ridc_restarted(from_workload(w), w.u0, w.dt, w.nsteps, 4, w.restart_every)
        errs[restarts] = np.linalg.norm(u - exact) / np.linalg.norm(exact)
    assert errs[10] < errs[0], errs


# ---------------------------------------------------------------- viscous Burgers
def test_burgers_flux_telescopes():
    """Flux form: the sum over the nodes of f^N leaves only the wall fluxes,
    sum_i f^N_i = -(u_n^2 - u_1^2) / (4 h)."""
    rng = np.random.default_rng(3)
    p = Burgers1DDirichlet(37, 1e-3)
    u = rng.standard_normal(37)
    assert np.sum(p.fN(u)) == pytest.approx(-(u[-1] ** 2 - u[0] ** 2) / (4 * p.h), rel=1e-12)


def test_burgers_flux_is_second_order():
    """f^N approximates -u u_x with an O(h^2) error for data that vanish at the walls."""
    errs = []
    for n in (99, 199, 399):
        p = Burgers1DDirichlet(n, 1e-3)
        x = np.arange(1, n + 1) * p.h
        u = np.sin(np.pi * x) + 0.3 * np.sin(2 * np.pi * x)
        ux = np.pi * np.cos(np.pi * x) + 0.6 * np.pi * np.cos(2 * np.pi * x)
        errs.append(np.max(np.abs(p.fN(u) + u * ux)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 3.6) & (ratios < 4.4)), ratios


@pytest.mark.parametrize("k", [1, 5, 40])
def test_dirichlet_laplacian_eigenpairs(k):
    n, nu = 63, 2e-3
    p = Burgers1DDirichlet(n, nu)
    x = np.arange(1, n + 1) * p.h
    q = np.sin(np.pi * k * x)
    lam = -4.0 / p.h ** 2 * np.sin(np.pi * k * p.h / 2) ** 2
    np.testing.assert_allclose(p.D(q), nu * lam * q, atol=1e-9 * abs(nu * lam))


def test_burgers_solve_matches_sine_transform():
    """(I - dt D)^{-1} is diagonal in the DST-I basis of the interior nodes."""
    n, nu, dt = 127, 1e-3, 0.01
    p = Burgers1DDirichlet(n, nu)
    r = np.random.default_rng(1).standard_normal(n)
    k = np.arange(1, n + 1)
    lam = -4.0 / p.h ** 2 * np.sin(np.pi * k * p.h / 2) ** 2
    want = scipy.fft.idst(scipy.fft.dst(r, type=1) / (1 - dt * nu * lam), type=1)
    np.testing.assert_allclose(p.solve(r, dt), want, atol=1e-13)


def test_burgers_is_fourth_order():
    """Theorem 1 with the Burgers nonlinearity: RIDC4 against the semi-discrete system
    integrated by scipy's DOP853 at tight tolerances (n = 199, T = 0.25)."""
    n, nu, T = 199, 1e-3, 0.25
    p = Burgers1DDirichlet(n, nu)
    x = np.arange(1, n + 1) * p.h
    u0 = np.sin(2 * np.pi * x) + 0.5 * np.sin(np.pi * x)
    ref = solve_ivp(lambda t, u: p.fN(u) + p.D(u), (0, T), u0, method="DOP853", rtol=1e-13,
                    atol=1e-14).y[:, -1]
    errs = []
    for nt in (100, 200, 400):
        u = ridc_sequential(p, u0, T / nt, nt, 4)
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 3.6), (errs, slopes)
