"""Semi-implicit RIDC-FBE in classic sequential IDC order (Section III), FP64.

Level 0 (predictor, eq. (pred) with linear f^S, i.e. eq. (imex_diffusion)):
    (I - dt D) eta0_{n+1} = eta0_n + dt f^N(eta0_n).
Level j >= 1 (corrector, eq. (corr)):
    (I - dt D) eta^j_{n+1} = eta^j_n + dt [f^N(eta^j_n) - f^N(eta^{j-1}_n)]
                             - dt D eta^{j-1}_{n+1}
                             + dt sum_i w[j][m][i] f(eta^{j-1}_{b+i}),   f = D eta + f^N.
As printed, eq. (corr) subtracts f^N(eta^{j-1}_n) without the factor dt; the error
equation it discretises (eq. (error_eqn)) and consistency both need dt on the whole
bracket, which is the reading used here.

Every level runs over the whole interval before the next one starts; level j only reads
final values of level j-1, which is why the lagged pipeline must reproduce these
numbers. When the requested run is shorter than the start-up stencil (nsteps < order-1),
the lower levels run on to t_{order-1} so the top level's start-up nodes exist.
"""
from __future__ import annotations

import numpy as np

from .quadrature import stencil, weight_table


def fbe(problem, y0: np.ndarray, dt: float, nsteps: int) -> list[np.ndarray]:
    """First-order IMEX (forward-backward Euler) history eta_0..eta_nsteps (eq. (imex_diffusion))."""
    eta = [np.array(y0, dtype=np.float64, copy=True)]
    for n in range(nsteps):
        eta.append(problem.solve(eta[n] + dt * problem.fN(eta[n]), dt))
    return eta


def ridc_sequential(problem, y0: np.ndarray, dt: float, nsteps: int, order: int,
                    all_levels: bool = False):
    """RIDC of order `order` (predictor + order-1 correctors) from y0 over nsteps steps.

    Returns eta^{order-1}_{nsteps}, or with all_levels=True the list
    [eta^0_{nsteps}, ..., eta^{order-1}_{nsteps}].
    """
    if order < 1:
        raise ValueError("order >= 1")
    w = weight_table(order)
    n_low = max(nsteps, order - 1)
    prev = fbe(problem, y0, dt, nsteps if order == 1 else n_low)
    finals = [prev[nsteps]]
    for j in range(1, order):
        fN_prev = [problem.fN(e) for e in prev]
        F_prev = [fN_prev[i] + problem.D(prev[i]) for i in range(len(prev))]
        n_j = nsteps if j == order - 1 else n_low
        eta = [np.array(y0, dtype=np.float64, copy=True)]
        for n in range(n_j):
            b, m = stencil(j, n)
            quad = np.zeros_like(eta[0])
            for i in range(j + 1):
                quad += w[j][m][i] * F_prev[b + i]
            rhs = (eta[n] + dt * (problem.fN(eta[n]) - fN_prev[n])
                   - dt * problem.D(prev[n + 1]) + dt * quad)
            eta.append(problem.solve(rhs, dt))
        finals.append(eta[nsteps])
        prev = eta
    return finals if all_levels else finals[-1]


def ridc_restarted(problem, y0: np.ndarray, dt: float, nsteps: int, order: int,
                   restart_every: int):
    """RIDC with restarts (Section III-E): the interval is cut into pieces of `restart_every`
    steps (the last piece may be shorter), and each piece is a fresh RIDC computation whose
    initial value is the most corrected solution at the end of the previous piece.
    restart_every <= 0 means no restarts. Returns the most corrected solution at nsteps."""
    if restart_every <= 0:
        return ridc_sequential(problem, y0, dt, nsteps, order)
    y = np.array(y0, dtype=np.float64, copy=True)
    done = 0
    while done < nsteps:
        k = min(restart_every, nsteps - done)
        y = ridc_sequential(problem, y, dt, k, order)
        done += k
    return y


def ridc_lagged(problem, y0: np.ndarray, dt: float, nsteps: int, order: int,
                with_schedule: bool = False):
    """The same RIDC, executed as the lagged pipeline of Section III-E: in every pipeline step
    each level that has its inputs advances by one time step, all of them reading only values
    that existed before the step. Level j computes eta^j_{n+1} from eta^{j-1}_{n+1} and the
    stencil nodes b..b+j of level j-1 (b = max(0, n+1-j)), so it may advance once level j-1
    has reached index max(n+1, j). Full histories are kept (no ring buffers): the identity
    with ridc_sequential is about values, and each update repeats its arithmetic exactly, so
    the two agree bit for bit.

    Returns eta^{order-1}_{nsteps}; with with_schedule=True also the list of level sets that
    advanced in each pipeline step.
    """
    if order < 1:
        raise ValueError("order >= 1")
    w = weight_table(order)
    n_low = max(nsteps, order - 1)
    last = [nsteps if (j == order - 1) else (nsteps if order == 1 else n_low)
            for j in range(order)]
    y = np.array(y0, dtype=np.float64, copy=True)
    eta = [[y.copy()] for _ in range(order)]
    fN = [[problem.fN(y)] for _ in range(order)]
    F = [[fN[j][0] + problem.D(y)] for j in range(order)]
    schedule = []
    while len(eta[order - 1]) - 1 < last[order - 1]:
        ready = []
        for j in range(order):
            n = len(eta[j]) - 1
            if n >= last[j]:
                continue
            if j == 0 or len(eta[j - 1]) - 1 >= max(n + 1, j):
                ready.append(j)
        if not ready:
            raise RuntimeError("pipeline stalled")
        new = {}
        for j in ready:                      # every update reads the state before this step
            n = len(eta[j]) - 1
            if j == 0:
                new[j] = problem.solve(eta[0][n] + dt * fN[0][n], dt)
                continue
            b, m = stencil(j, n)
            quad = np.zeros_like(y)
            for i in range(j + 1):
                quad += w[j][m][i] * F[j - 1][b + i]
            rhs = (eta[j][n] + dt * (fN[j][n] - fN[j - 1][n])
                   - dt * problem.D(eta[j - 1][n + 1]) + dt * quad)
            new[j] = problem.solve(rhs, dt)
        for j, e in new.items():
            eta[j].append(e)
            fN[j].append(problem.fN(e))
            F[j].append(fN[j][-1] + problem.D(e))
        schedule.append(ready)
    out = eta[order - 1][nsteps]
    return (out, schedule) if with_schedule else out
