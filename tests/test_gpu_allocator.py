"""Device memory through the caller's allocator (ridc_set_allocator), here torch's CUDA
caching allocator: results are bit for bit those of cudaMalloc'd buffers, every buffer goes
back to the allocator that made it, an allocation failure part-way through creation gives
back everything, misaligned pointers are refused, and the allocator cannot change while a
handle lives.
"""
import numpy as np
import pytest

import inputs
import oracle
from paper_1209_4297_gb300 import (Batch, Integrator, RidcError, set_allocator,
                                   use_torch_allocator)
from tests.gpu_util import need_cuda, rel_l2

pytestmark = pytest.mark.gpu

RIDC_ERR_OOM, RIDC_ERR_CUDA = -2, -3


@pytest.fixture(autouse=True)
def _default_allocator():
    yield
    set_allocator(None, None)


class Counting:
    """torch's caching allocator, with a record of what is out; optionally fails every
    request after the first `fail_after`, or hands out pointers moved by `offset` bytes."""

    def __init__(self, torch, fail_after=None, offset=0):
        self.torch, self.fail_after, self.offset = torch, fail_after, offset
        self.live, self.calls = {}, 0

    def alloc(self, nbytes, device):
        self.calls += 1
        if self.fail_after is not None and self.calls > self.fail_after:
            return None
        p = self.torch.cuda.caching_allocator_alloc(nbytes + self.offset, device=device)
        self.live[p + self.offset] = (p, nbytes)
        return p + self.offset

    def free(self, ptr, nbytes, device):
        base, n = self.live.pop(ptr)
        assert n == nbytes
        self.torch.cuda.caching_allocator_delete(base)


def _mixed_run(w, probe=None):
    with Integrator.from_workload(w, precision="mixed_bf16x3") as it:
        it.set_initial(w.u0)
        it.advance(w.nsteps)
        if probe:
            probe()
        return it.solution()


def test_torch_pool_gives_identical_results_and_gets_everything_back():
    torch = need_cuda()
    w = inputs.gray_scott_2d(n=256, nsteps=12, width=0.3)
    plain = _mixed_run(w)
    c = Counting(torch)
    set_allocator(c.alloc, c.free)
    base = torch.cuda.memory_allocated()
    seen = []
    got = _mixed_run(w, probe=lambda: seen.append(torch.cuda.memory_allocated() - base))
    np.testing.assert_array_equal(got, plain)
    assert c.calls >= 10 and not c.live, (c.calls, c.live)
    assert seen[0] > 0                               # torch held the library's buffers
    assert torch.cuda.memory_allocated() == base     # and got all of them back


def test_torch_pool_1d_with_schedule_growth_and_batch():
    """The 1D path re-allocates its schedule when a longer advance needs more room (the old
    buffer goes back only after the stream is idle); a batch allocates per instance."""
    torch = need_cuda()
    use_torch_allocator()
    base = torch.cuda.memory_allocated()
    w = inputs.adv_diff_1d(nsteps=64)
    with Integrator.from_workload(w) as it:
        it.set_initial(w.u0)
        for s in (2, 7, 55):   # each longer than the last
            it.advance(s)
        got = it.solution()
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, 64, w.order)
    assert rel_l2(got, ref) <= 1e-12
    ws = inputs.ensemble(6, nsteps=5)
    with Batch(ws, n_refine=1) as b:
        b.set_initial([x.u0[0] for x in ws])
        b.advance(5)
        pooled = [b.solution(i) for i in range(6)]
    assert torch.cuda.memory_allocated() == base
    use_torch_allocator(False)
    with Batch(ws, n_refine=1) as b:
        b.set_initial([x.u0[0] for x in ws])
        b.advance(5)
        for i in range(6):
            np.testing.assert_array_equal(b.solution(i), pooled[i])


@pytest.mark.parametrize("fail_after", [0, 3, 9])
def test_out_of_memory_part_way_gives_everything_back(fail_after):
    torch = need_cuda()
    w = inputs.gray_scott_2d(n=256, nsteps=2, width=0.3)
    c = Counting(torch, fail_after=fail_after)
    set_allocator(c.alloc, c.free)
    with pytest.raises(RidcError) as e:
        Integrator.from_workload(w, precision="mixed_fp16x3")
    assert e.value.code == RIDC_ERR_OOM
    assert not c.live


def test_misaligned_pointers_are_refused():
    torch = need_cuda()
    w = inputs.gray_scott_2d(n=64, nsteps=2, width=0.3)
    c = Counting(torch, offset=16)
    set_allocator(c.alloc, c.free)
    with pytest.raises(RidcError) as e:
        Integrator.from_workload(w)
    assert e.value.code == RIDC_ERR_CUDA
    assert not c.live


def test_allocator_cannot_change_while_a_handle_lives():
    need_cuda()
    w = inputs.gray_scott_2d(n=64, nsteps=2, width=0.3)
    with Integrator.from_workload(w):
        with pytest.raises(RidcError):
            use_torch_allocator()
    use_torch_allocator()   # no handle left: allowed
    with Integrator.from_workload(w) as it:
        it.set_initial(w.u0)
        it.advance(2)
        with pytest.raises(RidcError):
            use_torch_allocator(False)
