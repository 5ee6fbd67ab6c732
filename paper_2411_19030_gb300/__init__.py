"""GB300 (sm_103a) one-shot Parareal topology-optimisation pass for transient heat
conduction (arXiv 2411.19030): a C-ABI CUDA library (``include/ptg.h``,
``csrc/``) and its thin Python binding.

The library must be built (``build.build_library()``) before use; there is no CPU
fallback: every step of the pass runs in the library's CUDA kernels.
"""
from .api import (KIND_NAMES, Operator, PassBuffers, PTGError, SolveConfig, oneshot_pass, parareal_pass,
                  sequential_pass)
from ._ffi import (PTG_ADJOINT, PTG_FP32_REFINE, PTG_FP64, PTG_OBJ_MODIFIED, PTG_OBJ_POWER_MEAN, PTG_PARAREAL,
                   PTG_PLT, PTG_PRIMAL, PTG_SLICES_CHAINED, PTG_SLICES_PARALLEL)

__all__ = [
    "KIND_NAMES", "Operator", "PassBuffers", "PTGError", "SolveConfig", "oneshot_pass", "parareal_pass",
    "sequential_pass",
    "PTG_ADJOINT", "PTG_FP32_REFINE", "PTG_FP64", "PTG_OBJ_MODIFIED", "PTG_OBJ_POWER_MEAN", "PTG_PARAREAL",
    "PTG_PLT", "PTG_PRIMAL", "PTG_SLICES_CHAINED", "PTG_SLICES_PARALLEL",
]
