"""GB300-native semi-implicit RIDC (arXiv:1209.4297): Python binding of libridc.so.

The integrator runs entirely in the CUDA kernels of libridc.so (built in-tree for sm_103a by
`python -m paper_1209_4297_gb300.build`); this package only marshals arguments. Importing it
does not load the library; the first call does, and raises if the library is missing.
"""
from .binding import (Batch, Integrator, RidcError, debug_fail_alloc, error_string, lib,
                      quadrature_weights, set_allocator, use_torch_allocator,
                      schedule_plan, schedule_plan_from, schedule_plan_predictor, LIB_PATH,
                      KERNELS, PREDICTORS)

__all__ = ["Batch", "Integrator", "RidcError", "debug_fail_alloc", "error_string", "lib",
           "quadrature_weights", "set_allocator", "use_torch_allocator",
           "schedule_plan", "schedule_plan_from", "schedule_plan_predictor", "LIB_PATH",
           "KERNELS", "PREDICTORS"]
