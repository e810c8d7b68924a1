"""Pins of the oracle's 2D operators, solves and integrator.

  * Laplacian eigenpairs: cos(pi k (i+1/2)/N) (even ghost, Neumann) and sin(pi k (i+1/2)/N)
    (odd ghost, Dirichlet) with lambda_k = -(4/h^2) sin^2(pi k / 2N).
  * The spectral solve against dense Gaussian elimination of I - dt D on tiny grids.
  * Gray-Scott: (u, v) = (1, 0) is a fixed point; a uniform field follows the reaction ODE
    (the Laplacian of a constant vanishes under zero flux), compared with scipy's
    high-accuracy ODE integrator.
  * Gray-Scott with F = k = 0 and v = 0 is linear diffusion of u: one cosine mode under FBE
    follows (1 - dt Du lambda)^-n, and RIDC4 converges at order 4 to the matrix exponential.
  * Dirichlet advection-diffusion: pure diffusion of one sine mode under FBE is the
    closed form (1 - dt nu lambda)^-n; with advection, RIDC4 converges at order 4 to
    the matrix exponential of the semi-discrete system.
"""
import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import inputs
from oracle import AdvDiff2DDirichlet, GrayScott2DNeumann, fbe, ridc_sequential


def _lam(n, k):
    return -(4.0 * n * n) * np.sin(np.pi * k / (2 * n)) ** 2


@pytest.mark.parametrize("kx,ky", [(0, 0), (1, 0), (3, 5), (11, 15)])
def test_neumann_laplacian_eigenpairs(kx, ky):
    n = 16
    p = GrayScott2DNeumann(n, 1.0, 0.5, 0.04, 0.06)
    c = (np.arange(n) + 0.5) / n
    q = np.cos(np.pi * ky * c)[:, None] * np.cos(np.pi * kx * c)[None, :]
    got = p.D(np.stack([q, q]))
    lam = _lam(n, kx) + _lam(n, ky)
    np.testing.assert_allclose(got[0], lam * q, atol=1e-9 * (1 + abs(lam)))
    np.testing.assert_allclose(got[1], 0.5 * lam * q, atol=1e-9 * (1 + abs(lam)))


@pytest.mark.parametrize("kx,ky", [(1, 1), (2, 7), (16, 3), (16, 16)])
def test_dirichlet_laplacian_eigenpairs(kx, ky):
    n = 16
    p = AdvDiff2DDirichlet(n, 0.0, 0.0, 1.0)
    c = (np.arange(n) + 0.5) / n
    q = np.sin(np.pi * ky * c)[:, None] * np.sin(np.pi * kx * c)[None, :]
    lam = _lam(n, kx) + _lam(n, ky)
    np.testing.assert_allclose(p.D(q[None])[0], lam * q, atol=1e-9 * (1 + abs(lam)))


@pytest.mark.parametrize("kx,ky", [(1, 2), (5, 9)])
def test_dirichlet_central_advection_on_sine_modes(kx, ky):
    # the odd ghost continues sin(pi k x) exactly, so the central difference is exact on it
    n, a, b = 20, 0.6, -1.3
    p = AdvDiff2DDirichlet(n, a, b, 1.0)
    h = 1.0 / n
    c = (np.arange(n) + 0.5) / n
    sx, cx = np.sin(np.pi * kx * c), np.cos(np.pi * kx * c)
    sy, cy = np.sin(np.pi * ky * c), np.cos(np.pi * ky * c)
    q = sy[:, None] * sx[None, :]
    want = (-a * np.sin(np.pi * kx * h) / h * sy[:, None] * cx[None, :]
            - b * np.sin(np.pi * ky * h) / h * cy[:, None] * sx[None, :])
    np.testing.assert_allclose(p.fN(q[None])[0], want, atol=1e-11)


def _dense(p, shape):
    """The matrix of y -> D y, assembled column by column."""
    size = int(np.prod(shape))
    M = np.zeros((size, size))
    for col in range(size):
        e = np.zeros(size)
        e[col] = 1.0
        M[:, col] = p.D(e.reshape(shape)).ravel()
    return M


@pytest.mark.parametrize("cls", ["neumann", "dirichlet"])
@pytest.mark.parametrize("n", [5, 12, 24])
def test_spectral_solve_matches_dense_gaussian_elimination(cls, n):
    g = np.random.default_rng(n)
    if cls == "neumann":
        p = GrayScott2DNeumann(n, 2e-3, 1e-3, 0.04, 0.06)
        shape = (2, n, n)
    else:
        p = AdvDiff2DDirichlet(n, 0.3, 0.2, 5e-3)
        shape = (1, n, n)
    dt = 0.37
    A = np.eye(int(np.prod(shape))) - dt * _dense(p, shape)
    r = g.standard_normal(shape)
    want = np.linalg.solve(A, r.ravel()).reshape(shape)
    got = p.solve(r, dt)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-13


def test_gray_scott_fixed_point():
    n = 32
    p = GrayScott2DNeumann(n, 2e-5, 1e-5, 0.04, 0.06)
    y0 = np.stack([np.ones((n, n)), np.zeros((n, n))])
    y = ridc_sequential(p, y0, 0.5, 12, 4)
    np.testing.assert_allclose(y, y0, atol=1e-14)


def test_gray_scott_uniform_field_follows_reaction_ode_at_order_4():
    n, F, k = 8, 0.04, 0.06
    p = GrayScott2DNeumann(n, 2e-5, 1e-5, F, k)
    y0 = np.stack([np.full((n, n), 0.5), np.full((n, n), 0.25)])

    def rhs(t, y):
        u, v = y
        return [-u * v * v + F * (1 - u), u * v * v - (F + k) * v]

    T = 20.0
    ref = scipy.integrate.solve_ivp(rhs, (0, T), [0.5, 0.25], method="DOP853",
                                    rtol=1e-13, atol=1e-15).y[:, -1]
    errs = []
    for nt in (20, 40, 80):
        y = ridc_sequential(p, y0, T / nt, nt, 4)
        assert np.ptp(y[0]) < 1e-13 and np.ptp(y[1]) < 1e-13   # stays uniform
        errs.append(np.abs(y[:, 0, 0] - ref).max())
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert slopes.min() > 3.7, (errs, slopes)


def test_dirichlet_pure_diffusion_fbe_closed_form():
    n, nu, dt, steps, kx, ky = 16, 3e-3, 0.05, 9, 3, 2
    p = AdvDiff2DDirichlet(n, 0.0, 0.0, nu)
    c = (np.arange(n) + 0.5) / n
    q = (np.sin(np.pi * ky * c)[:, None] * np.sin(np.pi * kx * c)[None, :])[None]
    got = fbe(p, q, dt, steps)[-1]
    factor = (1.0 - dt * nu * (_lam(n, kx) + _lam(n, ky))) ** (-steps)
    np.testing.assert_allclose(got, factor * q, atol=1e-14)


@pytest.mark.parametrize("kx,ky", [(0, 0), (2, 1), (5, 7)])
def test_gray_scott_pure_diffusion_fbe_closed_form(kx, ky):
    """F = k = 0 and v = 0 leave u_t = Du Lap u: under FBE one cosine mode of u is scaled by
    (1 - dt Du (lambda_kx + lambda_ky))^-1 per step, and v stays exactly 0."""
    n, Du, Dv, dt, steps = 16, 2e-3, 1e-3, 0.5, 7
    p = GrayScott2DNeumann(n, Du, Dv, 0.0, 0.0)
    c = (np.arange(n) + 0.5) / n
    q = np.cos(np.pi * ky * c)[:, None] * np.cos(np.pi * kx * c)[None, :]
    y0 = np.stack([q, np.zeros((n, n))])
    got = fbe(p, y0, dt, steps)[-1]
    factor = (1.0 - dt * Du * (_lam(n, kx) + _lam(n, ky))) ** (-steps)
    np.testing.assert_allclose(got[0], factor * q, atol=1e-14)
    assert not np.any(got[1])


def test_gray_scott_linear_part_order_4_against_matrix_exponential():
    """With F = k = 0 and v = 0 the Gray-Scott system is linear diffusion of u: RIDC4 converges
    at order 4 to the matrix exponential of the semi-discrete Neumann Laplacian."""
    n, Du, T = 8, 5e-3, 4.0
    p = GrayScott2DNeumann(n, Du, 1e-3, 0.0, 0.0)
    g = np.random.default_rng(5)
    u0 = g.standard_normal((n, n))
    y0 = np.stack([u0, np.zeros((n, n))])
    M = np.zeros((n * n, n * n))
    for col in range(n * n):
        e = np.zeros((2, n, n))
        e[0].ravel()[col] = 1.0
        M[:, col] = p.D(e)[0].ravel()
    ref = (scipy.linalg.expm(T * M) @ u0.ravel()).reshape(n, n)
    errs = []
    for nt in (8, 16, 32):
        got = ridc_sequential(p, y0, T / nt, nt, 4)
        assert not np.any(got[1])
        errs.append(np.linalg.norm(got[0] - ref) / np.linalg.norm(ref))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert slopes[-1] > 3.7, (errs, slopes)


def test_dirichlet_adv_diff_order_4_against_matrix_exponential():
    w = inputs.adv_diff_2d(n=10, kmax=3)
    p = AdvDiff2DDirichlet(w.n, 0.8, -0.5, 2e-3)
    shape = w.u0.shape
    size = int(np.prod(shape))
    M = np.zeros((size, size))
    for col in range(size):
        e = np.zeros(size)
        e[col] = 1.0
        M[:, col] = (p.fN(e.reshape(shape)) + p.D(e.reshape(shape))).ravel()
    T = 0.5
    ref = (scipy.linalg.expm(T * M) @ w.u0.ravel()).reshape(shape)
    errs = []
    for nt in (40, 80, 160):
        errs.append(np.linalg.norm(ridc_sequential(p, w.u0, T / nt, nt, 4) - ref) / np.linalg.norm(ref))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert slopes[-1] > 3.7, (errs, slopes)
