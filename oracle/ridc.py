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
