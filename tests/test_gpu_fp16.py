"""The FP16 hi/lo split form of the mixed solve (RIDC_MIXED_FP16X3) through the C ABI.

An FP16 pair carries 22 significant bits against BF16's 16. One pass of either form is
also limited by the FP32 accumulation inside the tensor cores, an error common to both that
grows with the contraction length (N/2 per product): at N = 256 the split's representation
error still dominates and FP16 is about 3x more accurate per pass; at N >= 1024 the two
forms come within a factor of 1-3 of each other, near 1e-5 per pass, which bounds the bars
below (one pass <= 5e-5, one refinement <= 1e-9, two at the FP64 residual's floor).
FP16's exponent range is narrow, so every operand plane is scaled by its own power of two:
planes of very different magnitude in one batch, all-zero planes and consecutive solves of
different size must all keep the relative accuracy. Parity with the oracle keeps the mixed
bar (<= 1e-8 relative L2), and order 4 survives with a single refinement pass.
"""
import functools

import numpy as np
import pytest

import inputs
import oracle
from paper_1209_4297_gb300 import Integrator
from tests.gpu_util import need_cuda, rel_l2

pytestmark = pytest.mark.gpu


def _workload(kind, n):
    if kind == "neumann":
        return inputs.gray_scott_2d(n=n, nsteps=1)
    return inputs.adv_diff_2d(n=n, nsteps=1, kmax=2, nu=1e-3, dt=1.0 / 256)


def _rhs(n, planes, seed):
    """Smooth plus rough content, like a right-hand side in delta form."""
    g = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    smooth = np.sin(3 * x)[None, :, None] * np.cos(2 * x)[None, None, :]
    return smooth + 1e-3 * g.standard_normal((planes, n, n))


def _solve_errors(w, r, precision, n_refine):
    prob = oracle.from_workload(w)
    S = w.species
    with Integrator.from_workload(w, precision=precision, n_refine=n_refine) as it:
        got = it.solve_planes(r)
    return [rel_l2(got[p], prob.solve(np.stack([r[p]] * S), w.dt)[p % S])
            for p in range(r.shape[0])]


@pytest.mark.parametrize("kind", ["neumann", "dirichlet"])
@pytest.mark.parametrize("n_refine", [0, 1, 2])
@pytest.mark.parametrize("n", [256, 768])
def test_fp16_batched_solve_accuracy(kind, n_refine, n):
    need_cuda()
    w = _workload(kind, n)
    r = _rhs(n, 4 * w.species, 7)
    errs = _solve_errors(w, r, "mixed_fp16x3", n_refine)
    bar = {0: 5e-5, 1: 1e-9, 2: 1e-12}[n_refine]
    assert max(errs) <= bar, errs


@pytest.mark.parametrize("kind", ["neumann", "dirichlet"])
def test_fp16_pass_beats_bf16_pass(kind):
    """At N = 256 (short contractions) the split's own error dominates a pass: one FP16x3
    pass is at least 2x more accurate than one BF16x3 pass."""
    need_cuda()
    n = 256
    w = _workload(kind, n)
    r = _rhs(n, 4 * w.species, 11)
    e16 = max(_solve_errors(w, r, "mixed_fp16x3", 0))
    ebf = max(_solve_errors(w, r, "mixed_bf16x3", 0))
    assert e16 * 2 <= ebf, (e16, ebf)


def test_fp16_plane_scales_are_independent():
    """Planes from 1e-20 to 1e+20 in one batch (outside FP16's range without the per-plane
    scale), an all-zero plane, and a later solve of much smaller planes on the same handle
    (the maxima are reset per solve). The operands are staged in FP32, so the magnitudes
    stay inside its normal range."""
    need_cuda()
    n = 256
    w = _workload("neumann", n)
    prob = oracle.from_workload(w)
    r = _rhs(n, 8, 5)
    mags = [1e-20, 1e-12, 1.0, 1e6, 1e12, 1e20, 0.0, 3e-5]
    for p, m in enumerate(mags):
        r[p] *= m
    with Integrator.from_workload(w, precision="mixed_fp16x3", n_refine=1) as it:
        got = it.solve_planes(r)
        small = it.solve_planes(r * 1e-6)
    for p, m in enumerate(mags):
        want = prob.solve(np.stack([r[p]] * 2), w.dt)[p % 2]
        if m == 0.0:
            assert not np.any(got[p]) and not np.any(small[p]), p
            continue
        assert rel_l2(got[p], want) <= 1e-10, (p, rel_l2(got[p], want))
        assert rel_l2(small[p], want * 1e-6) <= 1e-10, (p, rel_l2(small[p], want * 1e-6))


def test_fp16_nonfinite_input_stays_visible():
    need_cuda()
    n = 256
    w = _workload("dirichlet", n)
    r = _rhs(n, 4, 2)
    r[1, 7, 9] = np.nan
    with Integrator.from_workload(w, precision="mixed_fp16x3", n_refine=1) as it:
        got = it.solve_planes(r)
    assert np.isnan(got[1]).any()
    prob = oracle.from_workload(w)
    for p in (0, 2, 3):   # the other planes are unaffected
        assert rel_l2(got[p], prob.solve(r[p][None], w.dt)[0]) <= 1e-10, p


def _run(w, precision, n_refine):
    with Integrator.from_workload(w, precision=precision, n_refine=n_refine) as it:
        it.set_initial(w.u0)
        it.advance(w.nsteps)
        return [it.level(j)[0] for j in range(w.order)]


@pytest.mark.parametrize("n_refine", [1, 2])
def test_gray_scott_fp16_matches_oracle_256(n_refine):
    need_cuda()
    w = inputs.gray_scott_2d(n=256, nsteps=30, width=0.3, seed=2)
    levels = _run(w, "mixed_fp16x3", n_refine)
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, w.nsteps, 4, all_levels=True)
    for j in range(4):
        assert rel_l2(levels[j], ref[j]) <= 1e-8, j


def test_dirichlet_fp16_matches_oracle_512():
    need_cuda()
    w = inputs.adv_diff_2d(n=512, nsteps=24, kmax=8, nu=1e-3)
    levels = _run(w, "mixed_fp16x3", 1)
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, w.nsteps, 4)
    assert rel_l2(levels[-1], ref) <= 1e-8


@functools.lru_cache(maxsize=1)
def _oracle_2048():
    w = inputs.gray_scott_2d(n=2048, nsteps=8)
    return w, oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, w.nsteps, 4,
                                     all_levels=True)


@pytest.mark.parametrize("n_refine", [1, 2])
def test_gray_scott_2048_fp16_full_size_truncated(n_refine):
    """The 2048^2 Gray-Scott workload in the FP16 form, start-up included."""
    need_cuda()
    w, ref = _oracle_2048()
    levels = _run(w, "mixed_fp16x3", n_refine)
    for j in range(4):
        assert rel_l2(levels[j], ref[j]) <= 1e-8, j


def test_fp16_keeps_order_4_with_one_refinement():
    need_cuda()
    w = inputs.adv_diff_2d(n=256, kmax=8, nu=1e-3)
    T, nts = 0.125, (16, 32, 64, 128)
    sols = []
    for nt in nts:
        with Integrator(w.kind, w.n, w.nu, T / nt, 4, a=w.a, b=w.b, precision="mixed_fp16x3",
                        n_refine=1) as it:
            it.set_initial(w.u0)
            it.advance(nt)
            sols.append(it.solution())
    diffs = [np.linalg.norm(sols[i] - sols[i + 1]) for i in range(len(sols) - 1)]
    slopes = np.log2(np.array(diffs[:-1]) / np.array(diffs[1:]))
    assert slopes[-1] > 3.7, (slopes, diffs)


def test_fp16_state_round_trip_with_bf16():
    """The saved state is FP64 in every precision: a BF16x3 run continues in the FP16 form."""
    need_cuda()
    w = inputs.gray_scott_2d(n=256, nsteps=14, width=0.3, seed=3)
    with Integrator.from_workload(w, precision="mixed_bf16x3", n_refine=2) as it:
        it.set_initial(w.u0)
        it.advance(6)
        state = it.save_state()
    with Integrator.from_workload(w, precision="mixed_fp16x3", n_refine=2) as it2:
        it2.load_state(state)
        it2.advance(8)
        got = it2.solution()
    ref = oracle.ridc_sequential(oracle.from_workload(w), w.u0, w.dt, 14, 4)
    assert rel_l2(got, ref) <= 1e-8


def test_fp16_profiling_counts_split_launches():
    need_cuda()
    w = inputs.gray_scott_2d(n=256, nsteps=10, width=0.3, seed=1)
    with Integrator.from_workload(w, precision="mixed_fp16x3", n_refine=2) as it:
        it.set_profiling(True)
        it.set_initial(w.u0)
        it.advance(w.nsteps)
        split = it.kernel_stats("split_f16")
        res = it.kernel_stats("residual")
        rhs = it.kernel_stats("rhs")
    # one split per right-hand side and per refinement residual
    assert split[0] == rhs[0] + res[0] and split[0] > 0, (split, rhs, res)
