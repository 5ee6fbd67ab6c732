"""Helpers for the GPU parity tests: build the CUDA operator from the same problem
statement as the oracle, move arrays, and compare."""
from __future__ import annotations

import numpy as np
import torch

from oracle import Problem
from paper_2411_19030_gb300 import Operator, SolveConfig
from paper_2411_19030_gb300.build import build_library

FP64_TOL = 1e-10          # FP64 path: max-abs error / max-abs value of each field
MIXED_T_TOL = 1e-6        # FP32-CG + FP64 refinement: temperatures and objective
MIXED_G_TOL = 1e-5        # FP32-CG + FP64 refinement: sensitivities


def ensure_built():
    build_library()


def gpu_operator(prob: Problem, precision: str = "fp64", **solve_kw) -> Operator:
    mat = prob.material
    solve = SolveConfig(precision=precision, **solve_kw)
    return Operator(prob.nx, prob.ny, prob.h,
                    dict(k0=mat.k0, kmin=mat.kmin, pk=mat.pk, c0=mat.c0, cmin=mat.cmin, pc=mat.pc),
                    prob.Nt, prob.Ntau, prob.dt, prob.p, np.asarray(prob.dirichlet, np.uint8),
                    q_elem=prob.q_elem, q_time=prob.q_time, solve=solve,
                    objective="modified" if prob.modified_objective else "power_mean")


def dev(a) -> torch.Tensor:
    return torch.tensor(np.asarray(a, dtype=np.float64), dtype=torch.float64, device="cuda").contiguous()


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = float(np.max(np.abs(b))) if b.size else 0.0
    if scale == 0.0:
        return float(np.max(np.abs(a))) if a.size else 0.0
    return float(np.max(np.abs(a - b))) / scale


def assert_close(name, a, b, tol):
    e = rel_err(a, b)
    assert e <= tol, f"{name}: relative error {e:.3e} > {tol:.1e}"
    return e
