"""The C ABI on its own: a plain C99 program (no Python, no torch) creates a mixed-precision
Gray-Scott integrator, advances it with host buffers on the legacy default stream, and its
result matches the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import inputs
import oracle
from tests.gpu_util import need_cuda, rel_l2

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIBDIR = os.path.join(ROOT, "paper_1209_4297_gb300")


def test_c_program_runs_the_integrator(tmp_path):
    need_cuda()
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "gpu_run")
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                         "-I", os.path.join(ROOT, "include"),
                         os.path.join(ROOT, "tests", "c", "gpu_run.c"), "-o", exe,
                         "-L", LIBDIR, "-lridc", "-Wl,-rpath," + LIBDIR],
                        capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    w = inputs.gray_scott_2d(n=256, nsteps=12, width=0.3, seed=4)
    fin, fout = tmp_path / "u0.bin", tmp_path / "out.bin"
    w.u0.astype(np.float64).tofile(fin)
    run = subprocess.run([exe, str(fin), str(fout), str(w.nsteps)], capture_output=True,
                         text=True, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    data = np.fromfile(fout, dtype=np.float64)
    got, t = data[:-1].reshape(w.u0.shape), data[-1]
    assert t == pytest.approx(w.nsteps * w.dt)
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, w.nsteps, w.order)
    assert rel_l2(got, ref) <= 1e-8
