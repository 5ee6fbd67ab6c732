"""The coarse-step solves with the Krylov vectors in global memory and the geometric multigrid
V-cycle (ptg_solve.coarse_stream = 2): the batched coarse propagators G_pri / G_adj (a3) and the
correction sweeps (a4) as streamed kernels, FP64 CG preconditioned by one V(1,1)-cycle of
Galerkin levels.  Forced on small even grids here: the one-shot pass must match the oracle
(FP64 and mixed precision; conductivity SIMP and Table 1 materials, the modified objective, the
PLT pass with G = 0, one CTA per slice and several), match the on-chip path to the solver
tolerance, and the preconditioner must cut the coarse-step CG iterations far below Jacobi's."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp
from oracle import coarse_states_from_sequential, oneshot_pass as o_oneshot
from paper_2411_19030_gb300 import PassBuffers, oneshot_pass
from tests.gpu_helpers import FP64_TOL, MIXED_G_TOL, MIXED_T_TOL, assert_close, dev, ensure_built, gpu_operator, host
from tests.problems import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


CASES = {
    # three levels (40 x 24 -> 20 x 12 -> 10 x 6), Table 1 materials, the paper's load
    "table1_40x24": lambda: (make_problem(40, 24, Nt=24, Ntau=6, dt=0.6 / 24, material="table1", sink="left_wide",
                                          q_time=W.q_time_paper(24, 0.6 / 24)), W.rho_uniform(40, 24, 91, 0.05, 0.95)),
    # four levels, conductivity SIMP with the contrast of rho ~ U(0, 1)
    "simp_64": lambda: (make_problem(64, 64, Nt=32, Ntau=8, dt=1 / 32, material="simp_k", sink="left_wide"),
                        W.rho_uniform(64, 64, 92, 0.0, 1.0)),
    "modified_objective": lambda: (make_problem(48, 32, Nt=16, Ntau=8, dt=1 / 16, material="table1", sink="bottom",
                                                modified_objective=True), W.rho_uniform(48, 32, 93, 0.1, 0.9)),
    # more slices than SMs: one CTA per slice (block barriers only)
    "one_cta_per_slice": lambda: (make_problem(32, 32, Nt=160, Ntau=160, dt=1 / 160, material="simp_k",
                                               sink="left_wide"), W.rho_uniform(32, 32, 94, 0.2, 0.8)),
}


def run(prob, rho, U_old, V_old, precision, coarse_stream, plt=False):
    # rtol 1e-12 in FP64: on the modified-objective case (Table 1, dtau = 1/8) neither path reaches
    # 1e-13 within the refinement limit, the on-chip stepper included
    op = gpu_operator(prob, precision, rtol=1e-12 if precision == "fp64" else 1e-10, coarse_stream=coarse_stream)
    buf = PassBuffers(op)
    buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
    buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
    op.assemble(dev(rho))
    Theta, grad = oneshot_pass(op, buf, plt=plt) if plt else oneshot_pass(op, buf)
    torch.cuda.synchronize()
    return op, buf, Theta, grad


def _states(prob, rho, seed):
    rho_old = W.rho_warm_perturb(rho, seed=seed, amp=0.05)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    return U_old, V_old


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("name", list(CASES))
def test_streamed_coarse_solves_match_oracle(name, precision):
    prob, rho = CASES[name]()
    U_old, V_old = _states(prob, rho, 95)
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    op, buf, Theta, grad = run(prob, rho, U_old, V_old, precision, 2)
    for kind in (1, 2, 4, 5):                                  # the streamed plans ran
        assert op.plan(kind, prob.Ntau if kind in (1, 4) else 1)["nthreads"] == 512
    tol_t, tol_g = (FP64_TOL, FP64_TOL) if precision == "fp64" else (MIXED_T_TOL, MIXED_G_TOL)
    assert_close("G_T", host(buf.G_T), ref["G_pri_old"][0], tol_t)
    assert_close("G_theta", host(buf.G_th), ref["G_pri_old"][1], tol_t)
    assert_close("T_hist", host(buf.T_hist), ref["T_hist"], tol_t)
    assert_close("U_new", host(buf.U_T_new), ref["U"][0], tol_t)
    assert_close("Theta", host(Theta), [ref["Theta"]], tol_t)
    assert_close("G_lam", host(buf.G_l), ref["G_adj_old"][0], tol_g)
    assert_close("V_new", host(buf.V_l_new), ref["V"][0], tol_g)
    assert_close("g_new", host(buf.V_g_new), ref["V"][1], tol_g)
    assert_close("grad", host(grad), ref["grad"], tol_g)
    st = op.stats()
    assert st["status"] == 0, st
    # the on-chip path gives the same pass to the solver tolerance
    _, _, _, grad2 = run(prob, rho, U_old, V_old, precision, 1)
    assert_close("streamed vs on chip", host(grad), host(grad2), 1e-9 if precision == "fp64" else 1e-6)


def test_multigrid_cuts_the_coarse_step_iterations():
    prob, rho = CASES["simp_64"]()
    U_old, V_old = _states(prob, rho, 96)
    counts = {}
    for cs, tl in ((2, "threelevel"), (1, "none")):
        op = gpu_operator(prob, "fp64", rtol=1e-13, coarse_stream=cs, twolevel=tl, cg_iters_max=4000)
        buf = PassBuffers(op)
        buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
        buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
        op.assemble(dev(rho))
        op.reset_stats()
        oneshot_pass(op, buf)
        torch.cuda.synchronize()
        st = op.stats()
        assert st["status"] == 0
        counts[cs] = st["kind_cg_iters"][1] / st["kind_solves"][1]
    # one V-cycle per iteration against Jacobi: several times fewer coarse-step iterations
    assert counts[2] * 4 < counts[1], counts


def test_streamed_plt_pass_matches_oracle():
    # G = 0 (Sec. 7, Eq. 7.2): the streamed sweeps copy F
    prob, rho = CASES["table1_40x24"]()
    U_old, V_old = _states(prob, rho, 97)
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old, plt=True)
    op, buf, Theta, grad = run(prob, rho, U_old, V_old, "fp64", 2, plt=True)
    assert_close("T_hist", host(buf.T_hist), ref["T_hist"], FP64_TOL)
    assert_close("grad", host(grad), ref["grad"], FP64_TOL)
    assert op.stats()["status"] == 0


def test_streamed_coarse_path_is_deterministic():
    prob, rho = CASES["table1_40x24"]()
    U, V = _states(prob, rho, 98)
    a = run(prob, rho, U, V, "fp32_refine", 2)
    b = run(prob, rho, U, V, "fp32_refine", 2)
    assert np.array_equal(host(a[3]), host(b[3])) and np.array_equal(host(a[1].T_hist), host(b[1].T_hist))


def _coarse_plans(prob, coarse_stream):
    op = gpu_operator(prob, "fp32_refine", coarse_stream=coarse_stream)
    return [op.plan(kind, prob.Ntau if kind in (1, 4) else 1) for kind in (1, 2, 4, 5)]


def test_library_streams_coarse_solves_on_large_grids_only():
    # from 30000 nodes: 192 x 192 (37 249 nodes) streams, 128 x 128 (16 641) stays on chip
    for n in (256, 192):
        big = make_problem(n, n, Nt=16, Ntau=8, dt=1 / 16, material="simp_k", sink="left_wide")
        assert _coarse_plans(big, 0) == _coarse_plans(big, 2)
        assert all(p["nthreads"] == 512 for p in _coarse_plans(big, 0))
    small = make_problem(128, 128, Nt=16, Ntau=8, dt=1 / 16, material="simp_k", sink="left_wide")
    assert _coarse_plans(small, 0) == _coarse_plans(small, 1)
