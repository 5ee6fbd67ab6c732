"""ptg_sensitivities_noalloc: the sensitivity reduction for callers that may not allocate
device memory (their memory belongs to another allocator, or cudaMalloc would synchronise a
timed loop).  It must give the same gradient as ptg_sensitivities, whose partial sums live
in the op's allocated workspace, on consecutive calls that share its static scratch array.

This file is collected last so that a failure here leaves every other test already run."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp, sequential_pass as o_sequential
from paper_2411_19030_gb300 import _ffi
from tests.gpu_helpers import FP64_TOL, assert_close, dev, ensure_built, gpu_operator, host
from tests.problems import make_problem

pytestmark = pytest.mark.gpu


def _noalloc(lib, prob, rho_d, lam_d, j0, j1, T_d, hist_j0, grad_d):
    m = prob.material
    mat = _ffi.ptg_material(m.k0, m.kmin, m.pk, m.c0, m.cmin, m.pc)
    return lib.ptg_sensitivities_noalloc(prob.nx, prob.ny, prob.h, prob.Nt, prob.dt, ctypes.byref(mat),
                                         rho_d.data_ptr(), lam_d.data_ptr(), j0, j1, T_d.data_ptr(), hist_j0,
                                         T_d.shape[0], grad_d.data_ptr(), torch.cuda.current_stream().cuda_stream)


# (nx, ny, Nt, j0, j1): 130 steps make chunks of 3 steps with a last chunk of 1, so the carry of
# T_{j-1} inside a chunk and a short last chunk both run; the second case is smaller in every
# direction and runs after the first, so partial sums the first left in the shared array lie
# beyond what it reads, and its window starts at j0 = 4 (history rows 3..19 only).
CASES = [(14, 11, 130, 1, 130), (9, 7, 23, 4, 19)]


@pytest.mark.parametrize("material", ["table1", "simp_k"])
def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(material):
    ensure_built()
    lib = _ffi.load()
    for nx, ny, Nt, j0, j1 in CASES:
        prob = make_problem(nx, ny, Nt=Nt, Ntau=1, dt=1 / Nt, material=material, sink="left_wide",
                            q_time=W.q_time_paper(Nt, 1 / Nt))
        rho = W.rho_uniform(nx, ny, 12, 0.05, 0.95)
        seq = o_sequential(OracleOp(prob, rho))
        # the oracle's sensitivity sum over j0..j1 alone: g_{j0} - g_{j1+1} (Eq. 4.7, cumulative)
        want = seq["g"][j0] - seq["g"][j1 + 1]
        T_d = dev(seq["T_hist"][j0 - 1:j1 + 1])
        lam_d, rho_d = dev(seq["lam"][j0:j1 + 1]), dev(rho)
        op = gpu_operator(prob)
        op.assemble(rho_d)
        ref = op.zeros(prob.Ne)
        op.sensitivities(lam_d, j0, j1, T_d, ref, hist_j0=j0 - 1)
        ref_h = host(ref)
        assert_close(f"allocating entry point vs oracle ({nx}x{ny}, j {j0}..{j1})", ref_h, want, FP64_TOL)
        for call in range(2):
            g = op.zeros(prob.Ne)
            assert _noalloc(lib, prob, rho_d, lam_d, j0, j1, T_d, j0 - 1, g) == _ffi.PTG_OK, lib.ptg_last_error()
            assert_close(f"no-alloc call {call + 1} ({nx}x{ny}, j {j0}..{j1})", host(g), ref_h, FP64_TOL)
        op.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    ensure_built()
    lib = _ffi.load()
    n = 2048                                    # 4 Mi elements > PTG_NOALLOC_SCRATCH_DOUBLES
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    mat = _ffi.ptg_material(1.0, 1e-3, 3.0, 1.0, 1.0, 1.0)
    rc = lib.ptg_sensitivities_noalloc(n, n, 1.0 / n, 10, 0.1, ctypes.byref(mat), buf.data_ptr(), buf.data_ptr(),
                                       1, 10, buf.data_ptr(), 0, 11, buf.data_ptr(), None)
    assert rc == _ffi.PTG_EINVAL
    assert b"scratch" in lib.ptg_last_error()
