"""Seeded synthetic inputs for the five RIDC workloads.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's tests.
It holds no arithmetic of the time integrator: it only draws initial fields and
problem parameters from seeded numpy PCG64 generators and returns plain FP64 arrays
laid out row-major as [species][y][x] (2D) or [x] (1D).

Grids:
  * 1D periodic on [0, 1): nodes x_i = i / N.
  * 2D on [0, 1]^2 (Neumann or Dirichlet walls): cell centres x_i = (i + 1/2) / N.

Workloads (where the problem statement leaves a detail open, each generator's docstring
states the choice made):
  * adv_diff_1d      N=256, a=1, nu=0.01, RIDC order 4, dt=1/512, T=1.
  * adv_diff_upwind_1d  the paper's advection-diffusion run (dx=1/1000, T=40, upwind).
  * burgers_1d       the paper's viscous Burgers run (dx=1/1000, T=1, Dirichlet walls).
  * gray_scott_2d    N x N, Du=2e-5, Dv=1e-5, F=0.04, k=0.06, dt=0.5.
  * ensemble_2d      512 Dirichlet advection-diffusion instances of uneven size.
  * adv_diff_2d      4096 x 4096 Dirichlet advection-diffusion, a=b=1, nu=1e-3.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * np.pi


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Workload:
    """One synthetic problem instance: operator parameters, initial data and run length."""
    kind: str                 # "adv_diff_1d_periodic" | "adv_diff_1d_upwind_periodic" |
                              # "burgers_1d_dirichlet" | "gray_scott_2d_neumann" |
                              # "adv_diff_2d_dirichlet"
    n: int                    # grid points per side
    dt: float
    nsteps: int
    order: int
    nu: tuple                 # diffusion coefficient per species
    u0: np.ndarray            # [species][y][x] (2D) or [x] (1D), float64, C-contiguous
    a: float = 0.0            # advection velocity along x
    b: float = 0.0            # advection velocity along y
    F: float = 0.0            # Gray-Scott feed rate
    k: float = 0.0            # Gray-Scott kill rate
    restart_every: int = 0    # restart interval in steps (0: none)
    meta: dict = field(default_factory=dict)

    @property
    def species(self) -> int:
        return len(self.nu)

    @property
    def dim(self) -> int:
        return 1 if "_1d_" in self.kind else 2


def adv_diff_1d(n: int = 256, seed: int = 0, nsteps: int = 512, dt: float = 1.0 / 512,
                order: int = 4, a: float = 1.0, nu: float = 0.01) -> Workload:
    """u0 = sum_{k=1..8} A_k sin(2 pi k x + phi_k), A_k ~ N(0,1) 2^-k, phi_k ~ U[0, 2 pi)."""
    g = _rng(seed)
    amp = g.standard_normal(8) * 2.0 ** -np.arange(1, 9)
    phase = g.uniform(0.0, TWO_PI, 8)
    x = np.arange(n, dtype=np.float64) / n
    u0 = np.zeros(n)
    for kk in range(8):
        u0 += amp[kk] * np.sin(TWO_PI * (kk + 1) * x + phase[kk])
    return Workload("adv_diff_1d_periodic", n, dt, nsteps, order, (nu,), np.ascontiguousarray(u0),
                    a=a, meta={"modes": list(range(1, 9)), "amp": amp, "phase": phase})


def adv_diff_upwind_1d(n: int = 1000, nsteps: int = 4000, T: float = 40.0, order: int = 4,
                       a: float = -0.1, nu: float = 1e-3, restarts: int = 10) -> Workload:
    """The paper's advection-diffusion run: u_t = 0.1 u_x + 1e-3 u_xx (a = -0.1 here), periodic,
    dx = 1/1000, T = 40, u0 = 2 + sin(2 pi x), upwind advection, restarts splitting the run
    into `restarts` equal intervals (0: none). Deterministic: no random draw."""
    x = np.arange(n, dtype=np.float64) / n
    u0 = 2.0 + np.sin(TWO_PI * x)
    every = nsteps // restarts if restarts > 0 else 0
    return Workload("adv_diff_1d_upwind_periodic", n, T / nsteps, nsteps, order, (nu,),
                    np.ascontiguousarray(u0), a=a, restart_every=every)


def burgers_1d(n: int = 999, nsteps: int = 2000, T: float = 1.0, order: int = 4,
               nu: float = 1e-3) -> Workload:
    """The paper's viscous Burgers run: u_t + (u^2/2)_x = 1e-3 u_xx, u(0) = u(1) = 0,
    dx = 1/1000 (999 interior nodes), T = 1, u0 = sin(2 pi x) + sin(pi x) / 2, no restarts.
    Deterministic: no random draw."""
    x = np.arange(1, n + 1, dtype=np.float64) / (n + 1)
    u0 = np.sin(TWO_PI * x) + 0.5 * np.sin(np.pi * x)
    return Workload("burgers_1d_dirichlet", n, T / nsteps, nsteps, order, (nu,),
                    np.ascontiguousarray(u0))


def gray_scott_2d(n: int = 1024, seed: int = 0, nsteps: int = 2000, dt: float = 0.5,
                  order: int = 4, Du: float = 2e-5, Dv: float = 1e-5, F: float = 0.04,
                  k: float = 0.06, width: float = 0.1, noise: float = 0.01) -> Workload:
    """u = 1, v = 0 with a `width`-wide square of (u, v) = (0.5, 0.25) whose centre is
    uniform in [w/2, 1 - w/2]^2; every cell value of both species is then multiplied by
    (1 + noise * U[-1, 1])."""
    g = _rng(seed)
    cx, cy = g.uniform(width / 2, 1.0 - width / 2, 2)
    x = (np.arange(n, dtype=np.float64) + 0.5) / n
    inx = np.abs(x - cx) <= width / 2
    iny = np.abs(x - cy) <= width / 2
    sq = iny[:, None] & inx[None, :]
    u = np.ones((n, n))
    v = np.zeros((n, n))
    u[sq] = 0.5
    v[sq] = 0.25
    y0 = np.stack([u, v])
    y0 *= 1.0 + noise * g.uniform(-1.0, 1.0, size=y0.shape)
    return Workload("gray_scott_2d_neumann", n, dt, nsteps, order, (Du, Dv), np.ascontiguousarray(y0),
                    F=F, k=k, meta={"centre": (float(cx), float(cy))})


def gray_scott_smooth(n: int = 256, seed: int = 0, nsteps: int = 16, dt: float = 1.0,
                      order: int = 4, Du: float = 2e-5, Dv: float = 1e-5, F: float = 0.04,
                      k: float = 0.06, width2: float = 0.02) -> Workload:
    """Smooth Gray-Scott data for convergence-order checks: a Gaussian bump
    g = exp(-|x - c|^2 / width2), centre uniform in [0.4, 0.6]^2; u = 1 - g/2, v = g/4."""
    g = _rng(seed)
    cx, cy = g.uniform(0.4, 0.6, 2)
    x = (np.arange(n, dtype=np.float64) + 0.5) / n
    bump = np.exp(-((x[:, None] - cy) ** 2 + (x[None, :] - cx) ** 2) / width2)
    y0 = np.stack([1.0 - 0.5 * bump, 0.25 * bump])
    return Workload("gray_scott_2d_neumann", n, dt, nsteps, order, (Du, Dv), np.ascontiguousarray(y0),
                    F=F, k=k, meta={"centre": (float(cx), float(cy))})


def _sine_field(n: int, coef: np.ndarray) -> np.ndarray:
    """sum_{ky,kx} coef[ky-1, kx-1] sin(pi kx x) sin(pi ky y) on the cell centres."""
    kmax = coef.shape[0]
    x = (np.arange(n, dtype=np.float64) + 0.5) / n
    s = np.sin(np.pi * np.arange(1, kmax + 1)[:, None] * x[None, :])   # [k][x]
    return s.T @ coef @ s                                                # [y][x]


def adv_diff_2d(n: int = 4096, seed: int = 0, nsteps: int = 512, dt: float | None = None,
                order: int = 4, a: float = 1.0, b: float = 1.0, nu: float = 1e-3,
                kmax: int = 16) -> Workload:
    """Low-mode field: coefficient N(0,1) / (kx^2 + ky^2) on sin(pi kx x) sin(pi ky y), kx, ky <= kmax."""
    g = _rng(seed)
    kk = np.arange(1, kmax + 1, dtype=np.float64)
    coef = g.standard_normal((kmax, kmax)) / (kk[:, None] ** 2 + kk[None, :] ** 2)
    u0 = _sine_field(n, coef)[None]
    if dt is None:
        dt = 1.0 / n
    return Workload("adv_diff_2d_dirichlet", n, dt, nsteps, order, (nu,), np.ascontiguousarray(u0),
                    a=a, b=b)


ENSEMBLE_SIDES = (64, 96, 128, 192, 256)


def ensemble_instance(i: int, nsteps: int = 256) -> Workload:
    """Instance i of the batched ensemble, drawn from seed 1000 + i: side ~ U{64..256},
    (a, b) ~ U[-1, 1]^2, nu ~ logU[1e-4, 1e-2], order ~ U{2, 3, 4}, dt = 1/(4 side);
    u0 = sum_{kx,ky<=4} N(0,1) 2^-(kx+ky) sin(pi kx x) sin(pi ky y)."""
    g = _rng(1000 + i)
    side = int(g.choice(ENSEMBLE_SIDES))
    a, b = g.uniform(-1.0, 1.0, 2)
    nu = float(10.0 ** g.uniform(-4.0, -2.0))
    order = int(g.choice((2, 3, 4)))
    kk = np.arange(1, 5, dtype=np.float64)
    coef = g.standard_normal((4, 4)) * 2.0 ** -(kk[:, None] + kk[None, :])
    u0 = _sine_field(side, coef)[None]
    return Workload("adv_diff_2d_dirichlet", side, 1.0 / (4 * side), nsteps, order, (nu,),
                    np.ascontiguousarray(u0), a=float(a), b=float(b), meta={"instance": i})


def ensemble(count: int = 512, nsteps: int = 256) -> list[Workload]:
    return [ensemble_instance(i, nsteps) for i in range(count)]


def by_name(name: str, **kw) -> Workload:
    """Named workloads at their full sizes; keyword overrides shrink them for tests."""
    if name == "adv_diff_1d":
        return adv_diff_1d(**kw)
    if name == "adv_diff_upwind_1d":
        return adv_diff_upwind_1d(**kw)
    if name == "burgers_1d":
        return burgers_1d(**kw)
    if name == "gray_scott_1024":
        return gray_scott_2d(**{"n": 1024, "nsteps": 2000, **kw})
    if name == "gray_scott_2048":
        return gray_scott_2d(**{"n": 2048, "nsteps": 1000, **kw})
    if name == "adv_diff_4096":
        return adv_diff_2d(**{"n": 4096, "nsteps": 512, **kw})
    raise KeyError(name)
