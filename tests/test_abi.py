"""The C ABI library loads, exports every entry point include/ridc.h declares, and its
host-only helpers behave (no GPU needed)."""
import os
import re
from fractions import Fraction

import numpy as np
import pytest

import paper_1209_4297_gb300 as R
from oracle.quadrature import lagrange_weights

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:int|void|long|const char\*)\s+(ridc_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = R.lib()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_error_strings():
    assert R.error_string(0) == "ok"
    assert "argument" in R.error_string(-1)
    assert R.error_string(-999) == "unknown error"


@pytest.mark.parametrize("order", [1, 2, 3, 4, 6, 8, 12])
def test_library_weights_match_exact_rationals(order):
    w = R.quadrature_weights(order)
    for j in range(1, order):
        for m in range(j):
            exact = lagrange_weights(j, m)
            for i in range(j + 1):
                want = float(exact[i])
                assert abs(w[j, m, i] - want) <= 2 * np.spacing(abs(want)) + 1e-300, (j, m, i)
            assert np.all(w[j, m, j + 1:] == 0)


def _simulate(order, nsteps, masks):
    """Replay a schedule: check every read of the rings hits a live value (ring j has j+3
    slots below the top level), and the start-up waits of Section III-E."""
    P = order
    p = [0] * P
    cap = [j + 3 if j < P - 1 else 2 for j in range(P)]
    # ring contents: slot -> time index held
    rings = [{0: 0} for _ in range(P)]
    first = [None] * P
    for s, m in enumerate(masks):
        adv = [(m >> j) & 1 for j in range(P)]
        for j in range(P):
            if not adv[j]:
                continue
            n = p[j]
            if first[j] is None:
                first[j] = s + 1
            if j > 0:
                b = max(0, n + 1 - j)
                need = set(range(b, b + j + 1)) | {n + 1, n}
                for t in need:
                    assert rings[j - 1].get(t % cap[j - 1]) == t, (s, j, t)
            assert rings[j].get(n % cap[j]) == n
        for j in range(P):
            if adv[j]:
                p[j] += 1
                rings[j][p[j] % cap[j]] = p[j]
    return p, first


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 8, 12])
@pytest.mark.parametrize("nsteps", [0, 1, 2, 3, 7, 40])
def test_schedule_reads_only_live_ring_slots(order, nsteps):
    masks = R.schedule_plan(order, nsteps)
    p, first = _simulate(order, nsteps, masks)
    assert p[order - 1] == nsteps
    for j in range(order - 1):
        assert p[j] == (max(nsteps, order - 1) if nsteps > 0 else 0)


@pytest.mark.parametrize("order", [2, 3, 4, 6, 8])
def test_startup_waits_and_steady_lag(order):
    """Level j first advances after waiting j(j+1)/2 steps; the run takes N + P(P-1)/2 steps
    and, once started, every level lags the one below by one step."""
    N = 60
    masks = R.schedule_plan(order, N)
    p, first = _simulate(order, N, masks)
    for j in range(order):
        assert first[j] == j * (j + 1) // 2 + 1
    assert len(masks) == N + order * (order - 1) // 2
    full = (1 << order) - 1
    steady = [s for s, m in enumerate(masks) if m == full]
    assert len(steady) >= N - order * order


def test_split_runs_schedule_the_same_steps():
    """Advancing 5 then 9 steps visits the same (level, index) pairs as advancing 14."""
    # host-side plan of one call is what ridc_advance replays; two calls = two plans from the
    # intermediate progress, which the C++ rule derives from p alone
    masks = R.schedule_plan(4, 14)
    pairs = []
    p = [0] * 4
    for m in masks:
        for j in range(4):
            if (m >> j) & 1:
                pairs.append((j, p[j]))
                p[j] += 1
    assert sorted(pairs) == sorted((j, n) for j in range(4) for n in range(p[j]))


def _reads_and_writes(order, p, m):
    """(slots read, slots written) per ring in one step with mask m from progress p."""
    P = order
    cap = [j + 3 if j < P - 1 else 2 for j in range(P)]
    reads = [set() for _ in range(P)]
    writes = [set() for _ in range(P)]
    for j in range(P):
        if not (m >> j) & 1:
            continue
        n = p[j]
        reads[j].add(n % cap[j])
        if j > 0:
            b = max(0, n + 1 - j)
            for t in set(range(b, b + j + 1)) | {n + 1, n}:
                reads[j - 1].add(t % cap[j - 1])
        writes[j].add((n + 1) % cap[j])
    return reads, writes


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 8, 12])
@pytest.mark.parametrize("splits", [[40], [1, 1, 1, 37], [3, 7, 30], [2, 5, 5, 28]])
def test_schedule_writes_never_hit_slots_read_in_the_same_step(order, splits):
    """Levels of one pipeline step may run concurrently (one CTA per level): a level's new
    slot must never be a slot that any level reads in that step, also across split advances."""
    P = order
    p = [0] * P
    top = 0
    for k in splits:
        top += k
        masks = R.schedule_plan_from(order, list(p), top)
        for m in masks:
            reads, writes = _reads_and_writes(order, p, int(m))
            for j in range(P):
                assert not (reads[j] & writes[j]), (order, p, int(m), j)
            for j in range(P):
                if (int(m) >> j) & 1:
                    p[j] += 1
        assert p[P - 1] == top


def test_fault_hooks_reject_bad_arguments():
    L = R.lib()
    assert L.ridc_debug_fail_alloc(-1) == -1
    assert L.ridc_debug_fail_alloc(0) == 0
    assert L.ridc_debug_stall_next_gemm(None) == -1


def test_allocator_hook_arguments():
    """ridc_set_allocator: both callbacks or neither (host-side checks, no device needed)."""
    from paper_1209_4297_gb300 import binding as B
    L = R.lib()
    assert L.ridc_set_allocator(B.ALLOC_FN(), B.FREE_FN(), None) == 0
    assert L.ridc_set_allocator(B.ALLOC_FN(lambda n, d, c: None), B.FREE_FN(), None) == -1
    assert L.ridc_set_allocator(B.ALLOC_FN(), B.FREE_FN(lambda p, n, d, c: None), None) == -1
    with pytest.raises(ValueError):
        B.set_allocator(lambda n, d: 0, None)
    B.set_allocator(None, None)


def test_binding_tables_match_the_header():
    """The ctypes binding's kind, precision and kernel-id tables agree with include/ridc.h."""
    from paper_1209_4297_gb300 import binding as B
    txt = open(os.path.join(ROOT, "include", "ridc.h")).read()
    enums = dict((k, int(v)) for k, v in re.findall(r"\b(RIDC_[A-Z0-9_]+)\s*=\s*(\d+)", txt))
    defines = dict((k, int(v)) for k, v in re.findall(r"#define\s+(RIDC_[A-Z0-9_]+)\s+(-?\d+)", txt))
    for name, val in B.KINDS.items():
        assert enums["RIDC_" + name.upper()] == val, name
    for name, val in B.PRECISIONS.items():
        assert enums["RIDC_" + name.upper()] == val, name
    ids = {"rhs": "RHS", "gemm_tc": "GEMM_TC", "gemm_f64": "GEMM_F64", "residual": "RESIDUAL",
           "finalize": "FINALIZE", "ridc1d": "1D", "split_f16": "SPLIT"}
    for name, val in B.KERNELS.items():
        assert defines["RIDC_KERNEL_" + ids[name]] == val, name
    assert len(B.KERNELS) == defines["RIDC_KERNEL_COUNT"]


# ---------------------------------------------------------------- schedules with an ARK predictor
P0 = {"fbe": 1, "ark3": 3, "ark4": 4}


def _simulate_p0(order, masks, p0):
    """Replay a schedule for a p0-th order predictor: corrector j reads the K = p0 + j node
    stencil t_b..t_{b+K-1}, b = max(0, n + 2 - K), of ring j-1 (p0 + j + 1 slots below the top
    level) plus eta^{j-1}_{n+1} and f^N(eta^{j-1}_n); every read must hit a live value."""
    P = order
    p = [0] * P
    cap = [p0 + j + 2 if j < P - 1 else 2 for j in range(P)]
    rings = [{0: 0} for _ in range(P)]
    first = [None] * P
    for s, m in enumerate(masks):
        reads = [set() for _ in range(P)]
        for j in range(P):
            if not (m >> j) & 1:
                continue
            n = p[j]
            if first[j] is None:
                first[j] = s + 1
            if j > 0:
                K = p0 + j
                b = max(0, n + 2 - K)
                need = set(range(b, b + K)) | {n + 1, n}
                for t in need:
                    assert rings[j - 1].get(t % cap[j - 1]) == t, (s, j, t)
                    reads[j - 1].add(t % cap[j - 1])
            assert rings[j].get(n % cap[j]) == n
            reads[j].add(n % cap[j])
        for j in range(P):
            if (m >> j) & 1:
                assert (p[j] + 1) % cap[j] not in reads[j], (s, j)   # no write over a read
        for j in range(P):
            if (m >> j) & 1:
                p[j] += 1
                rings[j][p[j] % cap[j]] = p[j]
    return p, first


@pytest.mark.parametrize("predictor", ["fbe", "ark3", "ark4"])
@pytest.mark.parametrize("order", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("nsteps", [0, 1, 2, 5, 30])
def test_predictor_schedule_reads_live_slots_and_waits(predictor, order, nsteps):
    p0 = P0[predictor]
    if p0 + order - 1 > 12:
        pytest.skip("beyond the widest stencil")
    masks = R.schedule_plan_predictor(order, predictor, nsteps)
    p, first = _simulate_p0(order, masks, p0)
    assert p[order - 1] == nsteps
    low = max(nsteps, p0 + order - 2) if order > 1 else nsteps
    for j in range(order - 1):
        assert p[j] == (low if nsteps > 0 else 0)
    if nsteps >= 5:
        for j in range(order):
            assert first[j] == 1 + j * (p0 - 1) + j * (j + 1) // 2, (j, first)


def test_predictor_schedule_fbe_is_the_paper_schedule():
    for order in (1, 2, 4, 8, 12):
        for nsteps in (0, 3, 17):
            np.testing.assert_array_equal(R.schedule_plan_predictor(order, "fbe", nsteps),
                                          R.schedule_plan(order, nsteps))


@pytest.mark.parametrize("predictor", ["ark3", "ark4"])
def test_predictor_schedule_split_and_limits(predictor):
    p0 = P0[predictor]
    order = 4
    p = [0] * order
    top = 0
    for k in (1, 2, 9, 20):
        top += k
        for m in R.schedule_plan_predictor(order, predictor, top, start=p):
            for j in range(order):
                if (int(m) >> j) & 1:
                    p[j] += 1
        assert p[order - 1] == top
    from paper_1209_4297_gb300 import RidcError
    with pytest.raises(RidcError):        # p0 + order - 1 > 12: no stencil that wide
        R.schedule_plan_predictor(13 - p0 + 1, predictor, 5)
    assert len(R.schedule_plan_predictor(13 - p0, predictor, 5)) > 0


def test_binding_predictors_match_the_header():
    from paper_1209_4297_gb300 import binding as B
    txt = open(os.path.join(ROOT, "include", "ridc.h")).read()
    enums = dict((k, int(v)) for k, v in re.findall(r"\b(RIDC_[A-Z0-9_]+)\s*=\s*(\d+)", txt))
    for name, val in B.PREDICTORS.items():
        assert enums["RIDC_PRED_" + name.upper()] == val, name
