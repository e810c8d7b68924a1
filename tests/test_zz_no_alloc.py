"""The batched FP64 solve that allocates nothing, checked against the handle-based solve.

Some callers cannot let a library call cudaMalloc. One example is a host code that reserves
all device memory for its own pool at start-up, where an extra allocation would fail or break
its memory budget. Another is a time-critical loop that cannot afford cudaMalloc/cudaFree,
which may synchronise the device. For them ridc_solve_planes_fixed works in a fixed device
array compiled into libridc.so. This file runs last so that, if it fails, a run that stops at
the first failure has already run every other test.
"""
import ctypes
from ctypes import POINTER, c_double, c_int, c_void_p

import numpy as np
import pytest

from paper_1209_4297_gb300 import Integrator, debug_fail_alloc, lib
from tests.gpu_util import need_cuda, rel_l2

pytestmark = pytest.mark.gpu

KIND = {"gray_scott_2d_neumann": 1, "adv_diff_2d_dirichlet": 2}


def _entry():
    f = lib().ridc_solve_planes_fixed
    f.restype = c_int
    f.argtypes = [c_int, c_int, POINTER(c_double), c_double, c_void_p, c_void_p, c_int, c_void_p]
    return f


def _call(f, kind, n, nu, dt, r_dev, out_dev, planes, stream):
    nu_arr = (c_double * len(nu))(*nu)
    return f(KIND[kind], n, nu_arr, dt, c_void_p(r_dev.data_ptr()), c_void_p(out_dev.data_ptr()),
             planes, c_void_p(stream))


@pytest.mark.parametrize("kind,n,planes,nu,dt", [
    ("gray_scott_2d_neumann", 96, 8, (2e-5, 1e-5), 0.5),
    ("adv_diff_2d_dirichlet", 128, 4, (1e-3,), 1.0 / 128),
])
def test_fixed_scratch_solve_matches_handle_solve_on_two_calls(kind, n, planes, nu, dt):
    torch = need_cuda()
    f = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    g = np.random.default_rng(11)
    inputs = [g.standard_normal((planes, n, n)), g.standard_normal((planes, n, n)) * 3.0 + 1.0]
    with Integrator(kind, n, nu, dt, 4) as it:
        wants = [it.solve_planes(r) for r in inputs]
    out = torch.empty((planes, n, n), dtype=torch.float64, device="cuda")
    for r, want in zip(inputs, wants):           # two calls in a row share the scratch array
        r_dev = torch.from_numpy(r).cuda()
        assert _call(f, kind, n, nu, dt, r_dev, out, planes, stream) == 0
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), want) <= 1e-13


def test_fixed_scratch_rejects_requests_beyond_its_capacity():
    torch = need_cuda()
    f = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    big = torch.zeros((1, 256, 256), dtype=torch.float64, device="cuda")
    assert _call(f, "adv_diff_2d_dirichlet", 256, (1e-3,), 0.01, big, big, 1, stream) == -6
    many = torch.zeros((9, 32, 32), dtype=torch.float64, device="cuda")
    assert _call(f, "adv_diff_2d_dirichlet", 32, (1e-3,), 0.01, many, many, 9, stream) == -6


def test_fixed_scratch_solve_in_place_allocates_nothing():
    """r and delta may be the same buffer; with the next device allocation armed to fail, the
    call still succeeds (it makes none) and the device's free memory does not change."""
    torch = need_cuda()
    f = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    kind, n, planes, nu, dt = "gray_scott_2d_neumann", 64, 6, (2e-5, 1e-5), 0.5
    r = np.random.default_rng(5).standard_normal((planes, n, n))
    with Integrator(kind, n, nu, dt, 4) as it:
        want = it.solve_planes(r)
    buf = torch.from_numpy(r).cuda()
    _call(f, kind, n, nu, dt, buf, buf, planes, stream)     # set-up call on this device
    torch.cuda.synchronize()
    buf.copy_(torch.from_numpy(r))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    debug_fail_alloc(1)
    try:
        rc = _call(f, kind, n, nu, dt, buf, buf, planes, stream)
        torch.cuda.synchronize()
    finally:
        debug_fail_alloc(0)
    assert rc == 0
    assert torch.cuda.mem_get_info()[0] == free0
    assert rel_l2(buf.cpu().numpy(), want) <= 1e-13
