"""ctypes binding of libridc.so (include/ridc.h): argument marshalling only.

Every step of the integrator runs in the library's CUDA kernels; this module converts numpy
arrays and torch tensors to pointers, passes the current torch CUDA stream, and turns
negative return codes into exceptions. There is no CPU fallback: if the shared library is
missing, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_long, c_size_t, c_uint, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libridc.so")

KINDS = {"adv_diff_1d_periodic": 0, "gray_scott_2d_neumann": 1, "adv_diff_2d_dirichlet": 2,
         "adv_diff_1d_upwind_periodic": 3, "burgers_1d_dirichlet": 4}
KINDS_1D = ("adv_diff_1d_periodic", "adv_diff_1d_upwind_periodic", "burgers_1d_dirichlet")
PRECISIONS = {"fp64": 0, "mixed_bf16x3": 1, "fp32_solve": 2, "mixed_fp16x3": 3}
PREDICTORS = {"fbe": 0, "ark3": 1, "ark4": 2}
KERNELS = {"rhs": 0, "gemm_tc": 1, "gemm_f64": 2, "residual": 3, "finalize": 4, "ridc1d": 5,
           "split_f16": 6}


class RidcError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} ({code})")


class Problem(ctypes.Structure):
    _fields_ = [("kind", c_int), ("a", c_double), ("b", c_double), ("F", c_double),
                ("k", c_double), ("precision", c_int), ("n_refine", c_int),
                ("restart_every", c_int), ("predictor", c_int)]


class Grid(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int)]


# allocator callbacks of ridc_set_allocator
ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_int, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_int, c_void_p)


_lib_handle = None


def lib() -> ctypes.CDLL:
    """The loaded libridc.so; raises if it has not been built."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1209_4297_gb300.build` (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz, lg = c_void_p, c_int, c_double, c_size_t, c_long
    sig = {
        "ridc_create": (i, [POINTER(Problem), POINTER(Grid), POINTER(c_double), d, i, vp,
                            POINTER(vp)]),
        "ridc_set_initial": (i, [vp, vp, sz, i]),
        "ridc_advance": (i, [vp, lg]),
        "ridc_get_solution": (i, [vp, vp, sz, i]),
        "ridc_get_level": (i, [vp, i, vp, sz, i, POINTER(lg)]),
        "ridc_get_time": (i, [vp, POINTER(d)]),
        "ridc_get_progress": (i, [vp, POINTER(lg), i]),
        "ridc_destroy": (None, [vp]),
        "ridc_error_string": (ctypes.c_char_p, [i]),
        "ridc_solve_planes": (i, [vp, vp, vp, i, i]),
        "ridc_save_state": (i, [vp, vp, POINTER(sz)]),
        "ridc_debug_fail_alloc": (i, [i]),
        "ridc_debug_stall_next_gemm": (i, [vp]),
        "ridc_load_state": (i, [vp, vp, sz]),
        "ridc_schedule_plan": (i, [i, lg, POINTER(c_uint), sz, POINTER(sz)]),
        "ridc_schedule_plan_from": (i, [i, POINTER(lg), lg, POINTER(c_uint), sz, POINTER(sz)]),
        "ridc_schedule_plan_predictor": (i, [i, i, POINTER(lg), lg, POINTER(c_uint), sz,
                                             POINTER(sz)]),
        "ridc_quadrature_weights": (i, [i, POINTER(c_double), sz]),
        "ridc_set_profiling": (i, [vp, i]),
        "ridc_get_kernel_stats": (i, [vp, i, POINTER(lg), POINTER(d)]),
        "ridc_launch_count": (lg, [vp]),
        "ridc_batch_create": (i, [i, POINTER(Problem), POINTER(Grid), POINTER(c_double),
                                  POINTER(c_double), POINTER(c_int), vp, POINTER(vp)]),
        "ridc_batch_set_initial": (i, [vp, POINTER(vp), i]),
        "ridc_batch_advance": (i, [vp, lg]),
        "ridc_batch_get_solution": (i, [vp, i, vp, sz, i]),
        "ridc_batch_cells": (lg, [vp]),
        "ridc_batch_autotune": (i, [vp, lg, POINTER(c_int), POINTER(ctypes.c_float)]),
        "ridc_batch_set_launch": (i, [vp, i]),
        "ridc_batch_tile_width": (i, [vp, i]),
        "ridc_batch_set_tile_width": (i, [vp, i, i]),
        "ridc_batch_graph_launches": (lg, [vp]),
        "ridc_batch_destroy": (None, [vp]),
        "ridc_set_allocator": (i, [ALLOC_FN, FREE_FN, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib_handle = L
    return L


def error_string(code: int) -> str:
    return lib().ridc_error_string(code).decode()


def _check(rc: int, where: str) -> None:
    if rc != 0:
        raise RidcError(rc, where)


def _ptr(x):
    """(pointer, count, on_device) of a C-contiguous float64 numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise TypeError("need a C-contiguous float64 array")
        return x.ctypes.data, x.size, 0
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError(type(x))
    if x.dtype != torch.float64 or not x.is_contiguous():
        raise TypeError("need a contiguous float64 tensor")
    return x.data_ptr(), x.numel(), int(x.is_cuda)


def _current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


# ---- host-only helpers ------------------------------------------------------------------
def schedule_plan(order: int, nsteps: int) -> np.ndarray:
    """Masks of the lock-step schedule of a fresh run (bit j: level j advances)."""
    cnt = c_size_t(0)
    L = lib()
    L.ridc_schedule_plan(order, nsteps, None, 0, byref(cnt))
    out = (c_uint * max(cnt.value, 1))()
    _check(L.ridc_schedule_plan(order, nsteps, out, cnt.value, byref(cnt)), "ridc_schedule_plan")
    return np.array(out[:cnt.value], dtype=np.uint32)


def schedule_plan_from(order: int, start, nsteps: int) -> np.ndarray:
    """Masks of the lock-step schedule continued from per-level progress `start` until the
    top level has taken nsteps steps."""
    st = (c_long * order)(*[int(v) for v in start])
    cnt = c_size_t(0)
    L = lib()
    L.ridc_schedule_plan_from(order, st, nsteps, None, 0, byref(cnt))
    out = (c_uint * max(cnt.value, 1))()
    _check(L.ridc_schedule_plan_from(order, st, nsteps, out, cnt.value, byref(cnt)),
           "ridc_schedule_plan_from")
    return np.array(out[:cnt.value], dtype=np.uint32)


def schedule_plan_predictor(order: int, predictor: str, nsteps: int, start=None) -> np.ndarray:
    """Masks of the lock-step schedule with predictor 'fbe', 'ark3' or 'ark4' (corrector j
    reads a p0 + j node stencil), from progress `start` (None: a fresh run)."""
    st = None if start is None else (c_long * order)(*[int(v) for v in start])
    cnt = c_size_t(0)
    L = lib()
    L.ridc_schedule_plan_predictor(order, PREDICTORS[predictor], st, nsteps, None, 0, byref(cnt))
    out = (c_uint * max(cnt.value, 1))()
    _check(L.ridc_schedule_plan_predictor(order, PREDICTORS[predictor], st, nsteps, out,
                                          cnt.value, byref(cnt)), "ridc_schedule_plan_predictor")
    return np.array(out[:cnt.value], dtype=np.uint32)


def debug_fail_alloc(k: int) -> None:
    """Test hook: the k-th device allocation from now on fails (0 disarms)."""
    _check(lib().ridc_debug_fail_alloc(k), "ridc_debug_fail_alloc")


_allocator_refs = None   # the installed callbacks must outlive every call that uses them


def set_allocator(alloc=None, free=None) -> None:
    """Route the library's device allocations through Python callables:
    alloc(nbytes, device) -> int device pointer (0 or None when out of memory) and
    free(ptr, nbytes, device). Both None: back to cudaMalloc / cudaFree. Raises while an
    Integrator or Batch exists."""
    global _allocator_refs
    if alloc is None and free is None:
        _check(lib().ridc_set_allocator(ALLOC_FN(), FREE_FN(), None), "ridc_set_allocator")
        _allocator_refs = None
        return
    if alloc is None or free is None:
        raise ValueError("give both alloc and free, or neither")

    def _a(nbytes, device, _ctx):
        try:
            return alloc(nbytes, device) or None
        except Exception:   # reported to the library as out of memory
            return None

    def _f(ptr, nbytes, device, _ctx):
        free(ptr, nbytes, device)

    refs = (ALLOC_FN(_a), FREE_FN(_f))
    _check(lib().ridc_set_allocator(refs[0], refs[1], None), "ridc_set_allocator")
    _allocator_refs = refs


def use_torch_allocator(enable: bool = True) -> None:
    """Let torch's CUDA caching allocator own the library's device memory (enable=False:
    cudaMalloc / cudaFree again). The library synchronises its stream before it returns a
    buffer, so torch may reuse it at once."""
    if not enable:
        set_allocator(None, None)
        return
    import torch

    def alloc(nbytes, device):
        return torch.cuda.caching_allocator_alloc(int(nbytes), device=int(device))

    def free(ptr, nbytes, device):
        torch.cuda.caching_allocator_delete(int(ptr))

    set_allocator(alloc, free)


def quadrature_weights(order: int) -> np.ndarray:
    """w[j][m][i] as computed by the library (exact rationals rounded to FP64)."""
    buf = (c_double * (order ** 3))()
    _check(lib().ridc_quadrature_weights(order, buf, order ** 3), "ridc_quadrature_weights")
    return np.array(buf[:], dtype=np.float64).reshape(order, order, order)


# ---- the integrator -----------------------------------------------------------------------
class Integrator:
    """One RIDC instance on the current CUDA device (see include/ridc.h)."""

    def __init__(self, kind: str, n: int, nu, dt: float, order: int, *, a: float = 0.0,
                 b: float = 0.0, F: float = 0.0, k: float = 0.0, precision: str = "fp64",
                 n_refine: int = 2, restart_every: int = 0, predictor: str = "fbe",
                 stream=None):
        L = lib()
        self._h = c_void_p(None)
        nu = np.atleast_1d(np.asarray(nu, dtype=np.float64))
        pr = Problem(KINDS[kind], a, b, F, k, PRECISIONS[precision], n_refine, restart_every,
                     PREDICTORS[predictor])
        gr = Grid(1 if kind in KINDS_1D else 2, n)
        if stream is None:
            stream = _current_stream()
        self.kind, self.n, self.order, self.dt = kind, n, order, dt
        self.species = 2 if kind == "gray_scott_2d_neumann" else 1
        self.shape = (n,) if gr.dim == 1 else (self.species, n, n)
        self.stream = stream
        _check(L.ridc_create(byref(pr), byref(gr), nu.ctypes.data_as(POINTER(c_double)), dt,
                             order, c_void_p(stream), byref(self._h)), "ridc_create")

    @classmethod
    def from_workload(cls, w, precision: str = "fp64", n_refine: int = 2, stream=None,
                      order: int | None = None, restart_every: int | None = None,
                      predictor: str = "fbe"):
        """Integrator for an inputs.Workload; restart_every defaults to the workload's."""
        return cls(w.kind, w.n, w.nu, w.dt, order or w.order, a=w.a, b=w.b, F=w.F, k=w.k,
                   precision=precision, n_refine=n_refine,
                   restart_every=(getattr(w, "restart_every", 0) if restart_every is None
                                  else restart_every), predictor=predictor, stream=stream)

    def close(self) -> None:
        if self._h:
            lib().ridc_destroy(self._h)
            self._h = c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_initial(self, u0) -> None:
        p, count, dev = _ptr(u0)
        _check(lib().ridc_set_initial(self._h, c_void_p(p), count, dev), "ridc_set_initial")

    def advance(self, nsteps: int) -> None:
        _check(lib().ridc_advance(self._h, nsteps), "ridc_advance")

    def solution(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        p, count, dev = _ptr(out)
        _check(lib().ridc_get_solution(self._h, c_void_p(p), count, dev), "ridc_get_solution")
        return out

    def level(self, j: int, out=None):
        if out is None:
            out = np.empty(self.shape)
        p, count, dev = _ptr(out)
        step = c_long(0)
        _check(lib().ridc_get_level(self._h, j, c_void_p(p), count, dev, byref(step)),
               "ridc_get_level")
        return out, step.value

    def progress(self) -> list[int]:
        buf = (c_long * self.order)()
        _check(lib().ridc_get_progress(self._h, buf, self.order), "ridc_get_progress")
        return list(buf)

    def time(self) -> float:
        t = c_double(0)
        _check(lib().ridc_get_time(self._h, byref(t)), "ridc_get_time")
        return t.value

    def debug_stall_next_gemm(self) -> None:
        """Test hook: the next tensor-core GEMM's bounded waits run out (RIDC_ERR_TIMEOUT)."""
        _check(lib().ridc_debug_stall_next_gemm(self._h), "ridc_debug_stall_next_gemm")

    def save_state(self) -> np.ndarray:
        """The whole integrator state (ridc_save_state) as a host byte array."""
        need = c_size_t(0)
        _check(lib().ridc_save_state(self._h, None, byref(need)), "ridc_save_state")
        buf = np.empty(need.value, dtype=np.uint8)
        _check(lib().ridc_save_state(self._h, c_void_p(buf.ctypes.data), byref(need)),
               "ridc_save_state")
        return buf

    def load_state(self, buf: np.ndarray) -> None:
        """Restore a state returned by save_state() of an integrator of the same problem."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().ridc_load_state(self._h, c_void_p(buf.ctypes.data), buf.size),
               "ridc_load_state")

    def solve_planes(self, r, out=None):
        """(I - dt nu_s L)^{-1} r for r of shape [planes][n][n] (plane p -> species p % S)."""
        if out is None:
            out = np.empty_like(r) if isinstance(r, np.ndarray) else r.new_empty(r.shape)
        pr, count, dev = _ptr(r)
        po, count2, dev2 = _ptr(out)
        if count != count2 or dev != dev2:
            raise ValueError("r and out must match in size and location")
        nplanes = count // (self.n * self.n)
        _check(lib().ridc_solve_planes(self._h, c_void_p(pr), c_void_p(po), nplanes, dev),
               "ridc_solve_planes")
        return out

    def set_profiling(self, enable) -> None:
        """False/0 off, True/1 every launch, k > 1 every launch of every k-th 2D step."""
        _check(lib().ridc_set_profiling(self._h, int(enable)), "ridc_set_profiling")

    def kernel_stats(self, name: str) -> tuple[int, float]:
        n = c_long(0)
        ms = c_double(0)
        _check(lib().ridc_get_kernel_stats(self._h, KERNELS[name], byref(n), byref(ms)),
               "ridc_get_kernel_stats")
        return n.value, ms.value

    def launch_count(self) -> int:
        return lib().ridc_launch_count(self._h)


class Batch:
    """An ensemble of independent 2D Dirichlet advection-diffusion instances (include/ridc.h,
    ridc_batch_*), advanced together by one persistent kernel launch per advance."""

    def __init__(self, workloads, n_refine: int = 0, stream=None):
        L = lib()
        self._h = c_void_p(None)
        n = len(workloads)
        probs = (Problem * n)(*[Problem(KINDS[w.kind], w.a, w.b, 0.0, 0.0, PRECISIONS["fp32_solve"],
                                        n_refine, 0, 0) for w in workloads])
        grids = (Grid * n)(*[Grid(2, w.n) for w in workloads])
        nu = (c_double * n)(*[w.nu[0] for w in workloads])
        dt = (c_double * n)(*[w.dt for w in workloads])
        order = (c_int * n)(*[w.order for w in workloads])
        if stream is None:
            stream = _current_stream()
        self.stream = stream
        self.sides = [w.n for w in workloads]
        _check(L.ridc_batch_create(n, probs, grids, nu, dt, order, c_void_p(stream),
                                   byref(self._h)), "ridc_batch_create")

    def close(self) -> None:
        if self._h:
            lib().ridc_batch_destroy(self._h)
            self._h = c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_initial(self, u0s) -> None:
        ptrs, dev = [], None
        for u in u0s:
            p, count, d = _ptr(u)
            dev = d if dev is None else dev
            if d != dev:
                raise ValueError("all initial fields on the host or all on the device")
            ptrs.append(p)
        arr = (c_void_p * len(ptrs))(*ptrs)
        _check(lib().ridc_batch_set_initial(self._h, arr, dev), "ridc_batch_set_initial")

    def advance(self, nsteps: int) -> None:
        _check(lib().ridc_batch_advance(self._h, nsteps), "ridc_batch_advance")

    def solution(self, i: int, out=None):
        if out is None:
            out = np.empty((self.sides[i], self.sides[i]))
        p, count, dev = _ptr(out)
        _check(lib().ridc_batch_get_solution(self._h, i, c_void_p(p), count, dev),
               "ridc_batch_get_solution")
        return out

    def cells(self) -> int:
        return lib().ridc_batch_cells(self._h)

    def graph_launches(self) -> int:
        """CUDA graphs launched so far (one per advance or autotuner trial)."""
        return lib().ridc_batch_graph_launches(self._h)

    def tile_width(self, side: int) -> int:
        """Half-columns per tensor-core tile of the products for grid side `side`."""
        rc = lib().ridc_batch_tile_width(self._h, side)
        _check(min(rc, 0), "ridc_batch_tile_width")
        return rc

    def set_tile_width(self, side: int, width: int) -> None:
        """Set that width: a multiple of 16 up to 64 that divides side/2."""
        _check(lib().ridc_batch_set_tile_width(self._h, side, width), "ridc_batch_set_tile_width")

    def set_launch(self, choice: int) -> None:
        """Launch shape CTAs per SM * 16 + cluster size, as autotune() reports it."""
        _check(lib().ridc_batch_set_launch(self._h, choice), "ridc_batch_set_launch")

    def autotune(self, nsteps: int = 4) -> tuple[int, float]:
        choice = c_int(0)
        ms = ctypes.c_float(0)
        _check(lib().ridc_batch_autotune(self._h, nsteps, byref(choice), byref(ms)),
               "ridc_batch_autotune")
        return choice.value, ms.value
