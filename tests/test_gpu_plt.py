"""The PLT variant (coarse propagators identically zero, Sec. 7) and the modified objective
Theta~ = Theta^p (Sec. 7.1) on the GPU, against the oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp
from oracle import coarse_states_from_sequential, objective_from_modified
from oracle import oneshot_pass as o_oneshot
from oracle import sequential_pass as o_sequential
from paper_2411_19030_gb300 import PassBuffers, oneshot_pass, sequential_pass
from paper_2411_19030_gb300.batch import Batch
from tests.gpu_helpers import (FP64_TOL, MIXED_G_TOL, MIXED_T_TOL, assert_close, dev, ensure_built, gpu_operator,
                               host)
from tests.problems import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def problem(name, modified=False):
    if name == "ragged_table1":      # non-square, capacity SIMP, time-varying load
        return make_problem(13, 9, Nt=24, Ntau=4, dt=1 / 24, material="table1", sink="left_wide",
                            q_time=W.q_time_paper(24, 1 / 24), modified_objective=modified), \
            W.rho_uniform(13, 9, 3, 0.05, 0.95)
    if name == "square40":           # several CTAs per slab, 8 slices
        return make_problem(40, Nt=64, Ntau=8, dt=1 / 64, modified_objective=modified), \
            W.rho_uniform(40, 40, 5, 0.2, 0.8)
    raise ValueError(name)


def run_oneshot(prob, rho, precision, plt, **kw):
    rho_old = W.rho_warm_perturb(rho, seed=77, amp=0.05)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old, plt=plt)
    op = gpu_operator(prob, precision, **kw)
    buf = PassBuffers(op)
    buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
    buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
    op.assemble(dev(rho))
    Theta, grad = oneshot_pass(op, buf, plt=plt)
    torch.cuda.synchronize()
    return op, buf, Theta, grad, ref


def check(buf, Theta, grad, ref, tol_t, tol_g):
    assert_close("F_T", host(buf.F_T), ref["F_pri"][0], tol_t)
    assert_close("U_new", host(buf.U_T_new), ref["U"][0], tol_t)
    assert_close("theta_new", host(buf.U_th_new), ref["U"][1], tol_t)
    assert_close("T_hist", host(buf.T_hist), ref["T_hist"], tol_t)
    assert_close("Theta", host(Theta), [ref["Theta"]], tol_t)
    assert_close("F_lam", host(buf.F_l), ref["F_adj"][0], tol_g)
    assert_close("V_lam", host(buf.V_l_new), ref["V"][0], tol_g)
    assert_close("V_g", host(buf.V_g_new), ref["V"][1], tol_g)
    assert_close("grad", host(grad), ref["grad"], tol_g)


@pytest.mark.parametrize("name", ["ragged_table1", "square40"])
@pytest.mark.parametrize("modified", [False, True])
def test_plt_pass_fp64_matches_oracle(name, modified):
    """Eq. 7.2 in the one-shot pass: u_{s+1} = F(u_s^old), v_s = F(v_{s+1}^old)."""
    prob, rho = problem(name, modified)
    op, buf, Theta, grad, ref = run_oneshot(prob, rho, "fp64", True)
    check(buf, Theta, grad, ref, FP64_TOL, FP64_TOL)
    # the corrections are copies of the fine results, bit for bit
    assert np.array_equal(host(buf.U_T_new)[1:], host(buf.F_T))
    assert np.array_equal(host(buf.V_l_new)[:-1], host(buf.F_l))
    assert op.stats()["status"] == 0
    assert op.stats()["by_kind"]["correct_primal"]["solves"] == 0
    assert op.stats()["by_kind"]["coarse_primal"]["solves"] == 0


@pytest.mark.parametrize("name", ["ragged_table1", "square40"])
def test_plt_pass_mixed_matches_oracle(name):
    prob, rho = problem(name, True)
    _, buf, Theta, grad, ref = run_oneshot(prob, rho, "fp32_refine", True, rtol=1e-10)
    check(buf, Theta, grad, ref, MIXED_T_TOL, MIXED_G_TOL)


@pytest.mark.parametrize("name", ["ragged_table1", "square40"])
def test_parareal_pass_with_modified_objective_matches_oracle(name):
    prob, rho = problem(name, True)
    _, buf, Theta, grad, ref = run_oneshot(prob, rho, "fp64", False)
    check(buf, Theta, grad, ref, FP64_TOL, FP64_TOL)


@pytest.mark.parametrize("name", ["ragged_table1", "square40"])
def test_sequential_modified_objective_and_conversion(name):
    """Sequential pass with Theta~ against the oracle, then the Sec. 7.1 conversion on the GPU
    against the oracle's conversion and against the power-mean pass of the same design."""
    prob_m, rho = problem(name, True)
    prob_t, _ = problem(name, False)
    ref_m = o_sequential(OracleOp(prob_m, rho))
    op_m, op_t = gpu_operator(prob_m), gpu_operator(prob_t)
    buf_m, buf_t = PassBuffers(op_m), PassBuffers(op_t)
    op_m.assemble(dev(rho)); op_t.assemble(dev(rho))
    Theta_m, grad_m = sequential_pass(op_m, buf_m)
    Theta_t, grad_t = sequential_pass(op_t, buf_t)
    torch.cuda.synchronize()
    assert_close("Theta~", host(Theta_m), [ref_m["Theta"]], FP64_TOL)
    assert_close("grad~", host(grad_m), ref_m["grad"], FP64_TOL)
    Theta_c = torch.empty(1, dtype=torch.float64, device="cuda")
    grad_c = torch.empty_like(grad_m)
    op_m.objective_from_modified(Theta_m, grad_m, Theta_c, grad_c)
    torch.cuda.synchronize()
    T_ref, g_ref = objective_from_modified(ref_m["Theta"], ref_m["grad"], prob_m.p)
    assert_close("Theta", host(Theta_c), [T_ref], FP64_TOL)
    assert_close("grad", host(grad_c), g_ref, FP64_TOL)
    assert_close("Theta vs power mean", host(Theta_c), host(Theta_t), FP64_TOL)
    assert_close("grad vs power mean", host(grad_c), host(grad_t), FP64_TOL)
    # in place (outputs aliasing the inputs)
    op_m.objective_from_modified(Theta_m, grad_m, Theta_m, grad_m)
    torch.cuda.synchronize()
    assert np.array_equal(host(Theta_m), host(Theta_c)) and np.array_equal(host(grad_m), host(grad_c))


def test_batched_plt_pass_matches_oracle_per_design():
    specs = [problem("ragged_table1", True), problem("square40", True),
             (make_problem(24, Nt=48, Ntau=6, dt=1 / 48, modified_objective=True), W.rho_uniform(24, 24, 9, 0.1, 0.9))]
    ops = [gpu_operator(p) for p, _ in specs]
    batch = Batch(ops)
    refs = []
    for d, (prob, rho) in enumerate(specs):
        rho_old = W.rho_warm_perturb(rho, seed=300 + d, amp=0.05)
        U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
        refs.append(o_oneshot(OracleOp(prob, rho), U_old, V_old, plt=True))
        b = batch.buffers(d)
        b["U_T"].copy_(dev(U_old[0])); b["U_theta"].copy_(dev(U_old[1]))
        b["V_lam"].copy_(dev(V_old[0])); b["V_g"].copy_(dev(V_old[1]))
        b["rho"].copy_(dev(rho))
    batch.assemble()
    batch.oneshot_pass(plt=True)
    torch.cuda.synchronize()
    for d, (prob, _) in enumerate(specs):
        b, ref = batch.buffers(d), refs[d]
        assert_close(f"T_hist[{d}]", host(b["T_hist"]), ref["T_hist"], FP64_TOL)
        assert_close(f"U_new[{d}]", host(b["U_T_new"]), ref["U"][0], FP64_TOL)
        assert_close(f"Theta[{d}]", host(b["U_theta_new"][prob.Ntau:]), [ref["Theta"]], FP64_TOL)
        assert_close(f"V_new[{d}]", host(b["V_lam_new"]), ref["V"][0], FP64_TOL)
        assert_close(f"grad[{d}]", host(b["V_g_new"][0]), ref["grad"], FP64_TOL)
