"""Failure detection without a GPU fault: allocation failures made on the host, and a
bounded device-side wait made to run out (a pipeline stage that is never loaded). Both must
end in a clean error code, leak nothing and leave the context usable."""
import numpy as np
import pytest

import inputs
import oracle
from paper_1209_4297_gb300 import Batch, Integrator, RidcError, debug_fail_alloc
from tests.gpu_util import need_cuda, rel_l2

pytestmark = pytest.mark.gpu

OOM, TIMEOUT = -2, -5


def _free_bytes(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _every_allocation_fails_cleanly(torch, make):
    """Arm the k-th allocation to fail for k = 1, 2, ... until creation no longer reaches it;
    each failed creation must report RIDC_ERR_OOM and give back every byte."""
    k, failures = 1, 0
    try:
        while True:
            before = _free_bytes(torch)
            debug_fail_alloc(k)
            try:
                obj = make()
            except RidcError as e:
                assert e.code == OOM, (k, e.code)
                assert _free_bytes(torch) == before, k
                failures += 1
                k += 1
                continue
            obj.close()
            break
    finally:
        debug_fail_alloc(0)
    return failures


def test_integrator_creation_survives_every_allocation_failure():
    torch = need_cuda()
    w = inputs.gray_scott_2d(n=256, nsteps=4, seed=1)
    n = _every_allocation_fails_cleanly(
        torch, lambda: Integrator.from_workload(w, precision="mixed_bf16x3"))
    assert n >= 20   # rings, work buffers, tables and operands
    with Integrator.from_workload(w, precision="mixed_bf16x3") as it:   # still works
        it.set_initial(w.u0)
        it.advance(4)
        got = it.solution()
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, 4, w.order)
    assert rel_l2(got, ref) <= 1e-8


def test_1d_and_batch_creation_survive_allocation_failures():
    torch = need_cuda()
    w1 = inputs.burgers_1d(n=300, nsteps=10, T=0.01)
    assert _every_allocation_fails_cleanly(torch, lambda: Integrator.from_workload(w1)) >= 8
    ws = [inputs.ensemble_instance(i, nsteps=4) for i in range(6)]
    assert _every_allocation_fails_cleanly(torch, lambda: Batch(ws)) >= 3


def test_gemm_wait_timeout_is_reported_and_the_context_recovers():
    need_cuda()
    w = inputs.gray_scott_2d(n=256, nsteps=4, seed=2)
    rng = np.random.default_rng(7)
    r = rng.standard_normal((4, 256, 256))
    prob = oracle.from_workload(w)
    with Integrator.from_workload(w, precision="mixed_bf16x3") as it:
        it.debug_stall_next_gemm()
        with pytest.raises(RidcError) as e:
            it.solve_planes(r)
        assert e.value.code == TIMEOUT
        got = it.solve_planes(r)   # the flag was cleared; the next solve is correct
    want = np.stack([prob.solve(r[2 * q: 2 * q + 2], w.dt) for q in range(2)]).reshape(r.shape)
    assert rel_l2(got, want) <= 1e-8
