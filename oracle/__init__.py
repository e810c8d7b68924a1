"""CPU FP64 oracle for semi-implicit RIDC-FBE (Ong, Melfi & Christlieb, arXiv:1209.4297).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package: only the
tests, the smoke check of the package entry module and the CPU-baseline leg of the
benchmark may use it. It shares no code with the CUDA path.

It runs the predictor and the correctors in classic sequential IDC order (every level
over the whole time interval before the next level starts), with the paper's direct
formulas: the FBE step of Section II, eq. (imex_diffusion) / eq. (pred), the corrector
eq. (corr) and the Lagrange quadrature of Section III-C. Implicit solves are exact
(dense LU in 1D; an orthonormal cosine/sine eigen-basis from scipy.fft in 2D).

The predictor is FBE (RIDC-FBE, Theorem 1) or one of the paper's third- and fourth-order
IMEX additive Runge-Kutta methods (oracle.ark; RIDC built on them is Theorem 2). The 1D
problems can also run in long double (dtype=np.longdouble), which measures the FP64
oracle's own rounding on long runs.

Pins (tests/test_oracle_*.py): exact rational quadrature weights against the textbook
Newton-Cotes / Adams-Moulton values, the semi-discrete Fourier solution of periodic
advection-diffusion, closed-form FBE amplification factors, observed order p under
dt halving (Theorem 1), dense Gaussian elimination on tiny grids, the discrete
eigenpairs of the Laplacians, the Gray-Scott fixed point and uniform-field ODE, and
a matrix-exponential solution of the 2D Dirichlet problem.
"""
from .quadrature import lagrange_weights, weight_table, stencil
from .problems import (AdvDiff1DPeriodic, AdvDiff1DUpwindPeriodic, Burgers1DDirichlet,
                       GrayScott2DNeumann, AdvDiff2DDirichlet, from_workload)
from .ridc import ridc_sequential, ridc_restarted, ridc_lagged, fbe, predict, quadrature_nodes
from .ark import ARK3, ARK4, TABLEAUX, ark_step, predictor_order

__all__ = ["lagrange_weights", "weight_table", "stencil", "AdvDiff1DPeriodic",
           "AdvDiff1DUpwindPeriodic", "Burgers1DDirichlet", "GrayScott2DNeumann",
           "AdvDiff2DDirichlet", "from_workload", "ridc_sequential", "ridc_restarted", "ridc_lagged", "fbe",
           "predict", "quadrature_nodes", "ARK3", "ARK4", "TABLEAUX", "ark_step", "predictor_order"]
