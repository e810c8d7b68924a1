"""include/ridc.h is a C header: a plain C99 program compiles against it, links to
libridc.so and calls the host-only entry points (no device is touched)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIBDIR = os.path.join(ROOT, "paper_1209_4297_gb300")


def test_c99_caller(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    if not os.path.exists(os.path.join(LIBDIR, "libridc.so")):
        pytest.skip("libridc.so not built")
    exe = str(tmp_path / "host_abi")
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                         "-I", os.path.join(ROOT, "include"),
                         os.path.join(ROOT, "tests", "c", "host_abi.c"), "-o", exe,
                         "-L", LIBDIR, "-lridc", "-Wl,-rpath," + LIBDIR],
                        capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "FAIL" not in run.stdout
