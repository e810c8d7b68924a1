"""Restarts (Section III-E) and checkpoint/resume of the CUDA path, through the C ABI.

Restarts: every `restart_every` steps of the most corrected level all levels restart from
its solution; parity with the oracle's restarted RIDC (FP64 <= 1e-12, mixed <= 1e-8).
Checkpoint/resume: a state saved by ridc_save_state and loaded into a fresh integrator
continues bit for bit like the saved one.
"""
import ctypes

import numpy as np
import pytest

import inputs
import oracle
from paper_1209_4297_gb300 import Integrator, RidcError, lib
from tests.gpu_util import need_cuda, rel_l2

pytestmark = pytest.mark.gpu


def _restarted(w, every, precision="fp64", order=None, splits=None):
    need_cuda()
    order = order or w.order
    with Integrator.from_workload(w, precision=precision, order=order,
                                  restart_every=every) as it:
        it.set_initial(w.u0)
        for s in (splits or [w.nsteps]):
            it.advance(s)
        return it.solution(), it.progress(), it.time()


@pytest.mark.parametrize("every", [1, 3, 7])
def test_1d_restarts_match_oracle(every):
    w = inputs.adv_diff_1d(n=64, nsteps=40, dt=1.0 / 256)
    got, prog, t = _restarted(w, every, splits=[13, 27])
    ref = oracle.ridc_restarted(oracle.from_workload(w), w.u0, w.dt, 40, w.order, every)
    assert rel_l2(got, ref) <= 1e-12
    # after the last restart time every level stands at it; the top level at 40
    assert prog[-1] == 40 and t == pytest.approx(40 * w.dt)
    assert all(p >= 40 - 40 % every for p in prog)


def test_1d_one_level_restarts_change_nothing():
    w = inputs.adv_diff_1d(n=64, nsteps=30, dt=1.0 / 256)
    plain, _, _ = _restarted(w, 0, order=1)
    for every in (1, 4):
        got, _, _ = _restarted(w, every, order=1, splits=[11, 19])
        np.testing.assert_array_equal(got, plain)


def test_gray_scott_fp64_restarts_match_oracle():
    w = inputs.gray_scott_2d(n=48, nsteps=17, width=0.3, seed=5)
    got, prog, _ = _restarted(w, 5, splits=[6, 11])
    ref = oracle.ridc_restarted(oracle.from_workload(w), w.u0, w.dt, 17, w.order, 5)
    assert rel_l2(got, ref) <= 1e-12
    assert prog[-1] == 17


def test_dirichlet_mixed_restarts_match_oracle():
    w = inputs.adv_diff_2d(n=256, nsteps=14)
    got, _, _ = _restarted(w, 6, precision="mixed_bf16x3")
    ref = oracle.ridc_restarted(oracle.from_workload(w), w.u0, w.dt, 14, w.order, 6)
    assert rel_l2(got, ref) <= 1e-8


def test_restart_split_is_bitwise_identical():
    w = inputs.gray_scott_2d(n=32, nsteps=20, width=0.3, seed=2)
    a, _, _ = _restarted(w, 4, splits=[20])
    b, _, _ = _restarted(w, 4, splits=[1, 3, 4, 5, 7])
    np.testing.assert_array_equal(a, b)


# ---------------------------------------------------------------- checkpoint / resume
def _resume_case(w, precision, split, every=0, load_precision=None):
    need_cuda()
    with Integrator.from_workload(w, precision=precision, restart_every=every) as it:
        it.set_initial(w.u0)
        it.advance(split)
        state = it.save_state()
        it.advance(w.nsteps - split)
        straight = it.solution()
        prog = it.progress()
    with Integrator.from_workload(w, precision=load_precision or precision,
                                  restart_every=every) as it2:
        it2.load_state(state)
        it2.advance(w.nsteps - split)
        return straight, it2.solution(), prog, it2.progress()


def test_resume_1d_is_bitwise_identical():
    w = inputs.adv_diff_1d(n=128, nsteps=50, dt=1.0 / 256)
    a, b, pa, pb = _resume_case(w, "fp64", 2)   # saved during start-up
    np.testing.assert_array_equal(a, b)
    assert pa == pb


def test_resume_gray_scott_mixed_is_bitwise_identical():
    w = inputs.gray_scott_2d(n=256, nsteps=16, seed=4)
    a, b, pa, pb = _resume_case(w, "mixed_bf16x3", 9)
    np.testing.assert_array_equal(a, b)
    assert pa == pb


def test_resume_across_restarts():
    w = inputs.gray_scott_2d(n=32, nsteps=21, width=0.3, seed=6)
    a, b, _, _ = _resume_case(w, "fp64", 7, every=5)
    np.testing.assert_array_equal(a, b)


def test_state_of_fp64_run_continues_in_mixed_precision():
    w = inputs.adv_diff_2d(n=256, nsteps=12)
    _, b, _, _ = _resume_case(w, "fp64", 6, load_precision="mixed_bf16x3")
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, 12, w.order)
    assert rel_l2(b, ref) <= 1e-8


def test_state_is_refused_by_another_problem():
    need_cuda()
    w = inputs.gray_scott_2d(n=32, nsteps=4, width=0.3, seed=1)
    with Integrator.from_workload(w) as it:
        with pytest.raises(RidcError):
            it.save_state()   # nothing to save before set_initial
        it.set_initial(w.u0)
        it.advance(3)
        state = it.save_state()
        L = lib()
        need = ctypes.c_size_t(0)
        assert L.ridc_save_state(it._h, None, ctypes.byref(need)) == 0
        assert need.value == state.size
        short = ctypes.c_size_t(need.value - 1)
        buf = np.empty(need.value, dtype=np.uint8)
        assert L.ridc_save_state(it._h, ctypes.c_void_p(buf.ctypes.data),
                                 ctypes.byref(short)) == -1
        assert short.value == need.value
        with pytest.raises(RidcError):
            it.load_state(state[:-8])   # truncated
        bad = state.copy()
        bad[0] ^= 1                      # not a state
        with pytest.raises(RidcError):
            it.load_state(bad)
    other = inputs.gray_scott_2d(n=32, nsteps=4, width=0.3, seed=1)
    with Integrator(other.kind, other.n, other.nu, other.dt * 0.5, other.order, F=other.F,
                    k=other.k) as it3:
        with pytest.raises(RidcError):
            it3.load_state(state)        # another dt
    with Integrator.from_workload(w, restart_every=2) as it4:
        with pytest.raises(RidcError):
            it4.load_state(state)        # another restart interval
