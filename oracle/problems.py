"""Method-of-lines problems y' = f^S(y) + f^N(y) with linear stiff part f^S = D y (Section II, eq. (ode)).

Each problem gives, in plain FP64 numpy:
  fN(y)         the explicit (non-stiff) term f^N,
  D(y)          the stiff term f^S(y) = D y, with D = nu * L per species (centred
                second differences, as in Section IV),
  solve(r, dt)  the exact solution y of (I - dt D) y = r  (eq. (imex_diffusion)).

Grids and boundary ghosts (the paper treats 1D periodic and 1D Dirichlet problems; the
2D cell-centred conventions are readings):
  * 1D periodic: x_i = i h, h = 1/N, neighbours wrap around.
  * 1D Dirichlet (Burgers): interior nodes x_i = i h, h = 1/(N+1), zero wall ghosts.
  * 2D Neumann:  cell centres (i + 1/2) h, even ghost u_{-1} = u_0, u_N = u_{N-1}.
  * 2D Dirichlet: cell centres, odd ghost u_{-1} = -u_0, u_N = -u_{N-1} (zero on the wall).
Arrays are [x] in 1D and [species][y][x] in 2D.

Extended precision (1D problems, dtype=np.longdouble): the same problem with its constants
and every operation in long double. The FP64 parameters (a, nu and h = 1/N rounded to FP64)
are converted exactly, so a long-double run evaluates the very algorithm the FP64 oracle runs
with a smaller rounding unit. Its implicit solve is mixed-precision iterative refinement
(Wilkinson): an FP64 LU solve, then `refine_passes` passes of x += LU^-1 (r - (I - dt D) x)
with the residual formed in long double. Each pass shrinks the error by about
cond(I - dt D) * 2^-53, so three passes reach the long-double rounding level for
cond <= 1e4 (mu = nu dt / h^2 up to about 2500).
"""
from __future__ import annotations

import numpy as np
import scipy.fft
import scipy.linalg


class _Solve1D:
    """Dense LU solve of (I - dt D) for the 1D problems, with the extended-precision
    refinement described in the module docstring when the right-hand side is long double."""
    refine_passes = 3

    def _scalar(self, v):
        # FP64 problems keep Python floats (the oracle's arithmetic); extended ones convert
        # the FP64 value exactly
        return float(v) if self.dtype == np.float64 else self.dtype.type(float(v))

    def _solve64(self, r: np.ndarray, dt: float) -> np.ndarray:
        # dense LU with partial pivoting of I - dt D, factored once per dt (in FP64)
        if dt not in self._lu:
            m = np.eye(self.n) - dt * self.matrix_D()   # long double for extended problems
            self._lu[dt] = scipy.linalg.lu_factor(np.asarray(m, dtype=np.float64))
        return scipy.linalg.lu_solve(self._lu[dt], r)

    def solve(self, r: np.ndarray, dt: float) -> np.ndarray:
        if r.dtype == np.float64:
            return self._solve64(r, dt)
        x = self._solve64(r.astype(np.float64), dt).astype(r.dtype)
        for _ in range(self.refine_passes):
            res = r - (x - dt * self.D(x))
            x = x + self._solve64(res.astype(np.float64), dt).astype(r.dtype)
        return x


class AdvDiff1DPeriodic(_Solve1D):
    """u_t + a u_x = nu u_xx on periodic [0,1): f^N = -a (u_{i+1} - u_{i-1}) / (2h), D = nu L."""

    def __init__(self, n: int, a: float, nu: float, dtype=np.float64):
        self.dtype = np.dtype(dtype)
        self.n = n
        self.a, self.nu = self._scalar(a), self._scalar(nu)
        self.h = self._scalar(1.0 / n)
        self._lu: dict[float, tuple] = {}

    def fN(self, u: np.ndarray) -> np.ndarray:
        return -self.a * (np.roll(u, -1) - np.roll(u, 1)) / (2.0 * self.h)

    def D(self, u: np.ndarray) -> np.ndarray:
        return self.nu * (np.roll(u, -1) - 2.0 * u + np.roll(u, 1)) / self.h ** 2

    def matrix_D(self) -> np.ndarray:
        """D as a dense FP64 matrix (the circulant of the periodic second difference)."""
        n = self.n
        L = np.zeros((n, n))
        for i in range(n):
            L[i, i] = -2.0
            L[i, (i + 1) % n] += 1.0
            L[i, (i - 1) % n] += 1.0
        return float(self.nu) * L / float(self.h) ** 2


class AdvDiff1DUpwindPeriodic(AdvDiff1DPeriodic):
    """The paper's advection-diffusion example (Section IV-A) on periodic [0,1): advection by
    first-order upwind differences, diffusion by centred differences. Written here as
    u_t + a u_x = nu u_xx (the paper's u_t = c u_x + d u_xx is a = -c, nu = d):
        a >= 0:  f^N_i = -a (u_i - u_{i-1}) / h,    a < 0:  f^N_i = -a (u_{i+1} - u_i) / h."""

    def fN(self, u: np.ndarray) -> np.ndarray:
        if self.a >= 0.0:
            return -self.a * (u - np.roll(u, 1)) / self.h
        return -self.a * (np.roll(u, -1) - u) / self.h


class Burgers1DDirichlet(_Solve1D):
    """Viscous Burgers, u_t + (u^2 / 2)_x = nu u_xx on [0,1] with u(0) = u(1) = 0 (Section
    IV-B). Unknowns at the n interior nodes x_i = i h, h = 1/(n+1), i = 1..n. The paper's
    numerical flux f_{i+1/2} = (u_{i+1}^2 + u_i^2) / 2 gives
        f^N_i = -(1/2) (f_{i+1/2} - f_{i-1/2}) / h,
    and D = nu L with the centred second difference; the wall values are the zero ghosts."""

    def __init__(self, n: int, nu: float, dtype=np.float64):
        self.dtype = np.dtype(dtype)
        self.n = n
        self.nu = self._scalar(nu)
        self.h = self._scalar(1.0 / (n + 1))
        self._lu: dict[float, tuple] = {}

    def _ghosted(self, u: np.ndarray) -> np.ndarray:
        z = np.zeros(1, dtype=u.dtype)
        return np.concatenate((z, u, z))

    def fN(self, u: np.ndarray) -> np.ndarray:
        g = self._ghosted(u)
        flux = 0.5 * (g[1:] ** 2 + g[:-1] ** 2)          # f_{i+1/2}, i = 0..n
        return -0.5 * (flux[1:] - flux[:-1]) / self.h

    def D(self, u: np.ndarray) -> np.ndarray:
        g = self._ghosted(u)
        return self.nu * (g[2:] - 2.0 * g[1:-1] + g[:-2]) / self.h ** 2

    def matrix_D(self) -> np.ndarray:
        """D as a dense FP64 matrix (zero wall ghosts)."""
        n = self.n
        L = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
        return float(self.nu) * L / float(self.h) ** 2


def _pad(u: np.ndarray, odd: bool) -> np.ndarray:
    """Pad the last two axes by one ghost cell: even (Neumann) or odd (Dirichlet) reflection."""
    p = np.pad(u, [(0, 0)] * (u.ndim - 2) + [(1, 1), (1, 1)], mode="edge")
    if odd:
        p[..., 0, :] *= -1.0
        p[..., -1, :] *= -1.0
        p[..., :, 0] *= -1.0
        p[..., :, -1] *= -1.0
    return p


def _lap2d(u: np.ndarray, h: float, odd: bool) -> np.ndarray:
    p = _pad(u, odd)
    return (p[..., 2:, 1:-1] + p[..., :-2, 1:-1] + p[..., 1:-1, 2:] + p[..., 1:-1, :-2]
            - 4.0 * u) / h ** 2


def _eig_neumann(n: int, h: float) -> np.ndarray:
    """Eigenvalues of the 1D Neumann cell-centred Laplacian, cosine modes k = 0..n-1."""
    k = np.arange(n)
    return -(4.0 / h ** 2) * np.sin(np.pi * k / (2 * n)) ** 2


def _eig_dirichlet(n: int, h: float) -> np.ndarray:
    """Eigenvalues of the 1D Dirichlet cell-centred Laplacian, sine modes k = 1..n."""
    k = np.arange(1, n + 1)
    return -(4.0 / h ** 2) * np.sin(np.pi * k / (2 * n)) ** 2


class _Separable2D:
    """Shared pieces of the two 2D problems: D = nu_s L with L the 5-point Laplacian."""
    odd = False

    def __init__(self, n: int, nu):
        self.n = n
        self.nu = np.asarray(nu, dtype=np.float64)
        self.h = 1.0 / n
        lam = _eig_dirichlet(n, self.h) if self.odd else _eig_neumann(n, self.h)
        self._lam2 = lam[:, None] + lam[None, :]          # [ky][kx]

    def D(self, y: np.ndarray) -> np.ndarray:
        return self.nu[:, None, None] * _lap2d(y, self.h, self.odd)

    def _fwd(self, y):
        f = scipy.fft.dstn if self.odd else scipy.fft.dctn
        return f(y, type=2, norm="ortho", axes=(-2, -1))

    def _inv(self, y):
        f = scipy.fft.idstn if self.odd else scipy.fft.idctn
        return f(y, type=2, norm="ortho", axes=(-2, -1))

    def solve(self, r: np.ndarray, dt: float) -> np.ndarray:
        # (I - dt nu_s L) is diagonal in the orthonormal cosine (Neumann) or sine
        # (Dirichlet) basis of type II: divide each mode by 1 - dt nu_s (lam_ky + lam_kx).
        den = 1.0 - dt * self.nu[:, None, None] * self._lam2[None]
        return self._inv(self._fwd(r) / den)


class GrayScott2DNeumann(_Separable2D):
    """u_t = Du lap u - u v^2 + F (1 - u),  v_t = Dv lap v + u v^2 - (F + k) v, zero-flux walls."""
    odd = False

    def __init__(self, n: int, Du: float, Dv: float, F: float, k: float):
        super().__init__(n, (Du, Dv))
        self.F, self.k = float(F), float(k)

    def fN(self, y: np.ndarray) -> np.ndarray:
        u, v = y[0], y[1]
        uvv = u * v * v
        return np.stack([-uvv + self.F * (1.0 - u), uvv - (self.F + self.k) * v])


class AdvDiff2DDirichlet(_Separable2D):
    """u_t + a u_x + b u_y = nu lap u, u = 0 on the walls; central advection differences."""
    odd = True

    def __init__(self, n: int, a: float, b: float, nu: float):
        super().__init__(n, (nu,))
        self.a, self.b = float(a), float(b)

    def fN(self, y: np.ndarray) -> np.ndarray:
        p = _pad(y, odd=True)
        ux = (p[..., 1:-1, 2:] - p[..., 1:-1, :-2]) / (2.0 * self.h)
        uy = (p[..., 2:, 1:-1] - p[..., :-2, 1:-1]) / (2.0 * self.h)
        return -self.a * ux - self.b * uy


def from_workload(w, dtype=np.float64) -> object:
    """Build the oracle problem for an inputs.Workload (dtype: 1D problems only)."""
    if w.kind == "adv_diff_1d_periodic":
        return AdvDiff1DPeriodic(w.n, w.a, w.nu[0], dtype)
    if w.kind == "adv_diff_1d_upwind_periodic":
        return AdvDiff1DUpwindPeriodic(w.n, w.a, w.nu[0], dtype)
    if w.kind == "burgers_1d_dirichlet":
        return Burgers1DDirichlet(w.n, w.nu[0], dtype)
    if np.dtype(dtype) != np.float64:
        raise ValueError("extended precision is provided for the 1D problems only")
    if w.kind == "gray_scott_2d_neumann":
        return GrayScott2DNeumann(w.n, w.nu[0], w.nu[1], w.F, w.k)
    if w.kind == "adv_diff_2d_dirichlet":
        return AdvDiff2DDirichlet(w.n, w.a, w.b, w.nu[0])
    raise KeyError(w.kind)
