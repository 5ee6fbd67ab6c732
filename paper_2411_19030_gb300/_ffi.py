"""ctypes binding of ``libptg.so`` (argument marshalling only; every computation runs in
the library's CUDA kernels).  The names are those of ``include/ptg.h``."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_longlong, c_void_p

from .build import library_path

PTG_OK, PTG_EINVAL, PTG_ENOCONV, PTG_ENONFINITE, PTG_ETIMEOUT, PTG_ECUDA, PTG_ENOMEM = 0, -1, -2, -3, -4, -5, -6
PTG_EBOUNDS = -7
PTG_FP64, PTG_FP32_REFINE, PTG_FP32_REFINE_ALL = 0, 1, 2
PTG_SLICES_PARALLEL, PTG_SLICES_CHAINED = 0, 1
PTG_PRIMAL, PTG_ADJOINT = 1, -1
PTG_OBJ_POWER_MEAN, PTG_OBJ_MODIFIED = 0, 1
PTG_PARAREAL, PTG_PLT = 0, 1
PTG_TWOLEVEL_NONE, PTG_TWOLEVEL_ADDITIVE, PTG_TWOLEVEL_VCYCLE, PTG_TWOLEVEL_THREELEVEL = 0, 1, 2, 3

ERROR_NAMES = {0: "PTG_OK", -1: "PTG_EINVAL", -2: "PTG_ENOCONV", -3: "PTG_ENONFINITE",
               -4: "PTG_ETIMEOUT", -5: "PTG_ECUDA", -6: "PTG_ENOMEM", -7: "PTG_EBOUNDS"}


class ptg_grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("h", c_double)]


class ptg_material(ctypes.Structure):
    _fields_ = [("k0", c_double), ("kmin", c_double), ("pk", c_double),
                ("c0", c_double), ("cmin", c_double), ("pc", c_double)]


class ptg_time(ctypes.Structure):
    _fields_ = [("Nt", c_int), ("Ntau", c_int), ("dt", c_double), ("p", c_double), ("objective", c_int)]


class ptg_solve(ctypes.Structure):
    _fields_ = [("precision", c_int), ("rtol", c_double), ("inner_rtol", c_double),
                ("cg_iters_max", c_int), ("refine_max", c_int), ("twolevel", c_int), ("grid_wide", c_int),
                ("smooth_steps", c_int), ("coarse_mesh", c_int),
                ("local_steps", c_int), ("initial_guess", c_int), ("fine_stream", c_int),
                ("coarse_stream", c_int)]


class ptg_stats(ctypes.Structure):
    _fields_ = [("status", c_int), ("fail_kind", c_int), ("fail_step", c_int), ("reserved", c_int),
                ("solves", c_longlong), ("cg_iters", c_longlong), ("refinements", c_longlong),
                ("max_cg_iters", c_longlong), ("kind_solves", c_longlong * 6), ("kind_cg_iters", c_longlong * 6),
                ("kind_refinements", c_longlong * 6)]


class ptg_pass_buffers(ctypes.Structure):
    _fields_ = [(n, c_void_p) for n in ("T_hist", "U_T", "U_theta", "V_lam", "V_g", "U_T_new", "U_theta_new",
                                        "V_lam_new", "V_g_new", "F_T", "F_theta", "G_T", "G_theta", "F_lam",
                                        "F_g", "G_lam", "G_g", "rho")]


_P = c_void_p   # device / host pointers and cudaStream_t are passed as addresses

SIGNATURES = {
    "ptg_version": (c_char_p, []),
    "ptg_last_error": (c_char_p, []),
    "ptg_op_create": (c_int, [POINTER(ptg_grid), POINTER(ptg_material), POINTER(ptg_time), POINTER(ptg_solve),
                              _P, _P, _P, c_int, POINTER(c_void_p)]),
    "ptg_op_destroy": (None, [_P]),
    "ptg_op_set_multigrid": (c_int, [_P, c_int, c_int, c_int]),
    "ptg_op_sizes": (c_int, [_P, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "ptg_op_get_plan": (c_int, [_P, c_int, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "ptg_op_set_plan": (c_int, [_P, c_int, c_int, c_int]),
    "ptg_fe_assemble_operator": (c_int, [_P, _P, _P]),
    "ptg_fine_propagate_slices": (c_int, [_P, c_int, c_int, c_int, _P, _P, _P, c_int, c_int, _P, _P, _P]),
    "ptg_coarse_sweep": (c_int, [_P, c_int, _P, _P, _P, _P, _P, _P, _P]),
    "ptg_coarse_sweep_slices": (c_int, [_P, c_int, c_int, c_int, _P, _P, _P, _P, _P, _P, _P]),
    "ptg_op_overlap_ok": (c_int, [_P, POINTER(c_int)]),
    "ptg_coarse_adjoint_split": (c_int, [_P, c_int, c_int, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ptg_coarse_adjoint_combine": (c_int, [_P, c_int, c_int, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ptg_parareal_correct": (c_int, [_P, c_int, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ptg_objective_from_modified": (c_int, [_P, _P, _P, _P, _P, _P]),
    "ptg_adjoint_sweep": (c_int, [_P, c_int, c_int, c_int, _P, c_int, c_int, _P, _P, _P, _P, _P, _P]),
    "ptg_sensitivities": (c_int, [_P, _P, c_int, c_int, _P, c_int, c_int, _P, _P]),
    "ptg_op_set_wait_limit": (c_int, [_P, ctypes.c_longlong]),
    "ptg_sensitivities_noalloc": (c_int, [c_int, c_int, c_double, c_int, c_double, POINTER(ptg_material), _P, _P,
                                          c_int, c_int, _P, c_int, c_int, _P, _P]),
    "ptg_batch_create": (c_int, [POINTER(c_void_p), c_int, POINTER(c_void_p)]),
    "ptg_batch_destroy": (None, [_P]),
    "ptg_batch_buffers": (c_int, [_P, c_int, POINTER(ptg_pass_buffers)]),
    "ptg_batch_assemble": (c_int, [_P, _P]),
    "ptg_batch_sequential_pass": (c_int, [_P, _P]),
    "ptg_batch_oneshot_pass": (c_int, [_P, c_int, _P]),
    "ptg_batch_commit": (c_int, [_P, _P]),
    "ptg_batch_run_phase": (c_int, [_P, c_int, _P]),
    "ptg_batch_set_plan": (c_int, [_P, c_int, c_int, c_int, c_int]),
    "ptg_batch_get_plan": (c_int, [_P, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "ptg_batch_design_path": (c_int, [_P, c_int, POINTER(c_int)]),
    "ptg_design_create": (c_int, [c_int, c_int, c_double, c_double, c_double, c_double, c_int, POINTER(c_void_p)]),
    "ptg_design_destroy": (None, [_P]),
    "ptg_design_forward": (c_int, [_P, _P, _P, _P, _P]),
    "ptg_design_backward": (c_int, [_P, _P, _P, _P, _P]),
    "ptg_design_volume": (c_int, [_P, _P, _P, _P]),
    "ptg_mma_create": (c_int, [c_int, c_double, c_double, c_double, POINTER(c_void_p)]),
    "ptg_mma_destroy": (None, [_P]),
    "ptg_mma_get_state": (c_int, [_P, POINTER(c_longlong), _P, _P, _P, _P]),
    "ptg_mma_set_state": (c_int, [_P, c_longlong, _P, _P, _P, _P]),
    "ptg_mma_update": (c_int, [_P, _P, c_double, _P, c_double, _P, _P]),
    "ptg_get_stats": (c_int, [_P, POINTER(ptg_stats)]),
    "ptg_reset_stats": (c_int, [_P, _P]),
}

_lib = None


def default_library() -> str:
    """The library ``load()`` opens: the build variant named by the environment variable
    PTG_LIBRARY ("release", the default, is libptg.so; "nvtx" libptg_nvtx.so; "debug"
    libptg_debug.so)."""
    return library_path(os.environ.get("PTG_LIBRARY") or "release")


def load(path: str | None = None):
    """Load the library (built by ``build.build_library``) and declare every signature.
    Raises OSError if the library is missing: there is no fallback implementation."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or default_library()
    if not os.path.exists(p):
        raise OSError(f"{p} is missing: run paper_2411_19030_gb300.build.build_library() first")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib
