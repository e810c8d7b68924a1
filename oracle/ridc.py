"""Semi-implicit RIDC in classic sequential IDC order (Section III), FP64.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; see the package docstring).

Level 0 (predictor). RIDC-FBE uses eq. (pred) with linear f^S, i.e. eq. (imex_diffusion):
    (I - dt D) eta0_{n+1} = eta0_n + dt f^N(eta0_n).
With predictor='ark3' or 'ark4', level 0 is instead the paper's third- or fourth-order IMEX
additive RK method of Section II (oracle.ark), which Theorem 2 allows in the prediction loop.
Level j >= 1 (corrector, eq. (corr)):
    (I - dt D) eta^j_{n+1} = eta^j_n + dt [f^N(eta^j_n) - f^N(eta^{j-1}_n)]
                             - dt D eta^{j-1}_{n+1}
                             + dt sum_i w[m][i] f(eta^{j-1}_{b+i}),   f = D eta + f^N.
As printed, eq. (corr) subtracts f^N(eta^{j-1}_n) without the factor dt; the error
equation it discretises (eq. (error_eqn)) and consistency both need dt on the whole
bracket, which is the reading used here.

Quadrature stencils (quadrature_nodes): corrector j of RIDC-FBE integrates level j-1 with
j+1 nodes (Section III-C). With a p0-th order predictor, level j-1 is accurate to order
p0 + j - 1 and corrector j must reach order p0 + j, so its interpolant needs p0 + j nodes:
the same sliding window, ending at t_{n+1} (or the fixed start-up window t_0.. before that),
one node per order gained.

Every level runs over the whole interval before the next one starts; level j only reads
final values of level j-1, which is why the lagged pipeline must reproduce these
numbers. When the requested run is shorter than the top level's start-up stencil, the lower
levels run on to its last node (t_{order-1} for RIDC-FBE) so the stencil's nodes exist.

dtype: np.float64 (the oracle), or np.longdouble for the extended-precision check of the
1D problems (their constants and every operation then run in long double, the implicit
solves by mixed-precision iterative refinement; see oracle.problems).
"""
from __future__ import annotations

import numpy as np

from .ark import TABLEAUX, ark_step, predictor_order
from .quadrature import lagrange_weights, stencil_nodes


def quadrature_nodes(j: int, predictor: str = "fbe") -> int:
    """Nodes of corrector j's quadrature stencil: j + 1 for RIDC-FBE (Section III-C), and
    p0 + j after a p0-th order predictor (the reading stated in the module docstring)."""
    return predictor_order(predictor) + j


def last_low_index(nsteps: int, order: int, predictor: str = "fbe") -> int:
    """Index the levels below the top run to: nsteps, or the last node of the top level's
    start-up stencil if that lies further (K - 1 with K = quadrature_nodes(order - 1))."""
    if order == 1:
        return nsteps
    return max(nsteps, quadrature_nodes(order - 1, predictor) - 1)


def _weights(K: int) -> list[list[float]]:
    """FP64 weights w[m][i] of the K-node stencil (node i at s = i, interval [m, m+1])."""
    return [[float(x) for x in lagrange_weights(K - 1, m)] for m in range(K - 1)]


def fbe(problem, y0: np.ndarray, dt: float, nsteps: int, dtype=np.float64) -> list[np.ndarray]:
    """First-order IMEX (forward-backward Euler) history eta_0..eta_nsteps (eq. (imex_diffusion))."""
    eta = [np.array(y0, dtype=dtype, copy=True)]
    for n in range(nsteps):
        eta.append(problem.solve(eta[n] + dt * problem.fN(eta[n]), dt))
    return eta


def predict(problem, y0: np.ndarray, dt: float, nsteps: int, predictor: str = "fbe",
            dtype=np.float64) -> list[np.ndarray]:
    """Level-0 history eta_0..eta_nsteps: FBE, or an ARK method of Section II."""
    if predictor == "fbe":
        return fbe(problem, y0, dt, nsteps, dtype)
    tab = TABLEAUX[predictor]
    eta = [np.array(y0, dtype=dtype, copy=True)]
    for n in range(nsteps):
        eta.append(ark_step(problem, eta[n], dt, tab))
    return eta


def _corrector_rhs(problem, dt, w, eta_j_n, fN_j_n, fN_prev_n, eta_prev_np1, F_prev, b, m, K):
    quad = np.zeros_like(eta_j_n)
    for i in range(K):
        quad += w[m][i] * F_prev[b + i]
    return (eta_j_n + dt * (fN_j_n - fN_prev_n) - dt * problem.D(eta_prev_np1) + dt * quad)


def ridc_sequential(problem, y0: np.ndarray, dt: float, nsteps: int, order: int,
                    all_levels: bool = False, predictor: str = "fbe", dtype=np.float64):
    """RIDC of order `order` (predictor + order-1 correctors) from y0 over nsteps steps.

    Returns eta^{order-1}_{nsteps}, or with all_levels=True the list
    [eta^0_{nsteps}, ..., eta^{order-1}_{nsteps}]. With an ARK predictor of order p0 the
    formal order is p0 + order - 1 (Theorem 2).
    """
    if order < 1:
        raise ValueError("order >= 1")
    n_low = last_low_index(nsteps, order, predictor)
    prev = predict(problem, y0, dt, n_low, predictor, dtype)
    finals = [prev[nsteps]]
    for j in range(1, order):
        K = quadrature_nodes(j, predictor)
        w = _weights(K)
        fN_prev = [problem.fN(e) for e in prev]
        F_prev = [fN_prev[i] + problem.D(prev[i]) for i in range(len(prev))]
        n_j = nsteps if j == order - 1 else n_low
        eta = [np.array(y0, dtype=dtype, copy=True)]
        for n in range(n_j):
            b, m = stencil_nodes(K, n)
            rhs = _corrector_rhs(problem, dt, w, eta[n], problem.fN(eta[n]), fN_prev[n],
                                 prev[n + 1], F_prev, b, m, K)
            eta.append(problem.solve(rhs, dt))
        finals.append(eta[nsteps])
        prev = eta
    return finals if all_levels else finals[-1]


def ridc_restarted(problem, y0: np.ndarray, dt: float, nsteps: int, order: int,
                   restart_every: int, predictor: str = "fbe", dtype=np.float64):
    """RIDC with restarts (Section III-E): the interval is cut into pieces of `restart_every`
    steps (the last piece may be shorter), and each piece is a fresh RIDC computation whose
    initial value is the most corrected solution at the end of the previous piece.
    restart_every <= 0 means no restarts. Returns the most corrected solution at nsteps."""
    if restart_every <= 0:
        return ridc_sequential(problem, y0, dt, nsteps, order, predictor=predictor, dtype=dtype)
    y = np.array(y0, dtype=dtype, copy=True)
    done = 0
    while done < nsteps:
        k = min(restart_every, nsteps - done)
        y = ridc_sequential(problem, y, dt, k, order, predictor=predictor, dtype=dtype)
        done += k
    return y


def ridc_lagged(problem, y0: np.ndarray, dt: float, nsteps: int, order: int,
                with_schedule: bool = False, predictor: str = "fbe"):
    """The same RIDC, executed as the lagged pipeline of Section III-E: in every pipeline step
    each level that has its inputs advances by one time step, all of them reading only values
    that existed before the step. Level j computes eta^j_{n+1} from eta^{j-1}_{n+1} and the
    K-node stencil b..b+K-1 of level j-1 (K = quadrature_nodes(j)), so it may advance once
    level j-1 has reached index max(n+1, K-1). Full histories are kept (no ring buffers): the
    identity with ridc_sequential is about values, and each update repeats its arithmetic
    exactly, so the two agree bit for bit.

    Returns eta^{order-1}_{nsteps}; with with_schedule=True also the list of level sets that
    advanced in each pipeline step.
    """
    if order < 1:
        raise ValueError("order >= 1")
    n_low = last_low_index(nsteps, order, predictor)
    last = [nsteps if j == order - 1 else n_low for j in range(order)]
    Ks = [quadrature_nodes(j, predictor) for j in range(order)]
    ws = [None] + [_weights(Ks[j]) for j in range(1, order)]
    tab = TABLEAUX.get(predictor)
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
            if j == 0 or len(eta[j - 1]) - 1 >= max(n + 1, Ks[j] - 1):
                ready.append(j)
        if not ready:
            raise RuntimeError("pipeline stalled")
        new = {}
        for j in ready:                      # every update reads the state before this step
            n = len(eta[j]) - 1
            if j == 0:
                if tab is None:
                    new[j] = problem.solve(eta[0][n] + dt * fN[0][n], dt)
                else:
                    new[j] = ark_step(problem, eta[0][n], dt, tab)
                continue
            b, m = stencil_nodes(Ks[j], n)
            rhs = _corrector_rhs(problem, dt, ws[j], eta[j][n], fN[j][n], fN[j - 1][n],
                                 eta[j - 1][n + 1], F[j - 1], b, m, Ks[j])
            new[j] = problem.solve(rhs, dt)
        for j, e in new.items():
            eta[j].append(e)
            fN[j].append(problem.fN(e))
            F[j].append(fN[j][-1] + problem.D(e))
        schedule.append(ready)
    out = eta[order - 1][nsteps]
    return (out, schedule) if with_schedule else out
