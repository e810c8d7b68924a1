"""Write the extended-precision reference solutions in tests/golden/extended_*.txt.

Each file holds the final solution of one FP64 workload recomputed by the CPU oracle with
every operation in long double (oracle.problems: 1D problems with dtype=np.longdouble; the
implicit solves by iterative refinement with long-double residuals). The algorithm, its
parameters and its initial data are those of the FP64 run, so the file is what that run
would produce without rounding error (to the long-double rounding level), and a comparison
with it measures rounding alone. Values are written rounded to FP64 (17 significant digits).

Calls only oracle/ and inputs/. Usage: python tests/golden/make_extended.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import inputs  # noqa: E402
import oracle  # noqa: E402


def cases():
    """name -> (workload, order, run); run(problem, dtype) returns the final solution."""
    out = {}
    # Section IV-B: viscous Burgers, 999 interior nodes, T = 1 in 2000 steps, RIDC-4
    w = inputs.burgers_1d()
    out["burgers_paper"] = (w, lambda p, d, w=w: oracle.ridc_sequential(
        p, w.u0, w.dt, w.nsteps, w.order, dtype=d))
    # Section IV-A: upwind advection-diffusion, N = 1000, T = 40 in 4000 steps, 10 restarts
    w = inputs.adv_diff_upwind_1d()
    out["upwind_paper"] = (w, lambda p, d, w=w: oracle.ridc_restarted(
        p, w.u0, w.dt, w.nsteps, w.order, w.restart_every, dtype=d))
    # RIDC-12 on periodic central advection-diffusion, n = 256, mu = nu dt / h^2 = 1, 70 steps
    w = inputs.adv_diff_1d(n=256, nsteps=70, dt=0.25 / 256, nu=4.0 / 256)
    out["order12_n256"] = (w, lambda p, d, w=w: oracle.ridc_sequential(
        p, w.u0, w.dt, w.nsteps, 12, dtype=d))
    return out


def path(name: str) -> str:
    return os.path.join(HERE, f"extended_{name}.txt")


def load(name: str) -> np.ndarray:
    return np.loadtxt(path(name), dtype=np.float64, comments="#")


def main():
    if np.finfo(np.longdouble).eps > 1e-18:
        raise SystemExit("long double is not wider than FP64 on this machine")
    for name, (w, run) in cases().items():
        ext = run(oracle.from_workload(w, np.longdouble), np.longdouble)
        with open(path(name), "w") as f:
            f.write(f"# {name}: final solution of the FP64 workload recomputed in long double "
                    f"(eps {np.finfo(np.longdouble).eps:.3e}) by the oracle; "
                    "tests/golden/make_extended.py\n")
            for v in np.asarray(ext, dtype=np.float64):
                f.write(f"{float(v)!r}\n")
        print(name, len(ext))


if __name__ == "__main__":
    main()
