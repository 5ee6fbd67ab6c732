"""GPU parity: every entry point of the C ABI against the CPU oracle, element by element,
on the same seeded inputs.  FP64 path: relative error <= 1e-10 of each field's max-abs
value; FP32-CG + FP64-refinement path: <= 1e-6 on temperatures and objective, <= 1e-5 on
sensitivities."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp
from oracle import coarse_states_from_sequential, oneshot_pass as o_oneshot, sequential_pass as o_sequential
from oracle.parareal import parareal as o_parareal
from paper_2411_19030_gb300 import PTG_ADJOINT, PTG_PRIMAL, PassBuffers, PTGError, oneshot_pass, sequential_pass
from tests.gpu_helpers import (FP64_TOL, MIXED_G_TOL, MIXED_T_TOL, assert_close, dev, ensure_built, gpu_operator,
                               host)
from tests.problems import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def case_problem(name):
    """Small problems that span several CTAs with ragged slabs and every code path."""
    if name == "ragged_table1":      # non-square, capacity SIMP active, time-varying load
        return make_problem(13, 9, Nt=24, Ntau=4, dt=1 / 24, material="table1", sink="left_wide",
                            q_time=W.q_time_paper(24, 1 / 24)), W.rho_uniform(13, 9, 3, 0.05, 0.95)
    if name == "plain32":            # the plain FP64 workload: 32x32, 100 steps, dt = 1e-3
        return make_problem(32, Nt=100, Ntau=10, dt=1e-3), W.rho_plain(32, 32, 0)
    if name == "paper_p20":          # Table 1, bottom sink, p = 20, Eq. 5.1 load
        return make_problem(20, Nt=30, Ntau=5, dt=1 / 30, material="table1", sink="bottom", p=20.0,
                            q_time=W.q_time_paper(30, 1 / 30)), np.full(400, 0.3)
    if name == "m1":                 # M = 1: every coarse step equals a fine step
        return make_problem(8, 7, Nt=6, Ntau=6, dt=0.05, material="table1", sink="left_wide"), \
            W.rho_uniform(8, 7, 5, 0.1, 0.9)
    if name == "one_slice":          # Ntau = 1
        return make_problem(9, Nt=8, Ntau=1, dt=0.05, sink="left_wide"), W.rho_uniform(9, 9, 6, 0.1, 0.9)
    if name == "tiny":               # smallest grid: 2 x 3 elements
        return make_problem(2, 3, Nt=4, Ntau=2, dt=0.1, material="table1", sink="left_wide"), \
            W.rho_uniform(2, 3, 7, 0.1, 0.9)
    raise KeyError(name)


CASES = ["ragged_table1", "plain32", "paper_p20", "m1", "one_slice", "tiny"]


@pytest.mark.parametrize("name", CASES)
def test_sequential_pass_fp64(name):
    """Initialisation of Alg. 3 (chained F_pri and F_adj) vs the oracle's sequential pass."""
    prob, rho = case_problem(name)
    oop = OracleOp(prob, rho)
    seq = o_sequential(oop)
    (U_T, U_th), (V_l, V_g), _ = coarse_states_from_sequential(oop, seq)
    op = gpu_operator(prob)
    buf = PassBuffers(op)
    op.assemble(dev(rho))
    Theta, grad = sequential_pass(op, buf)
    assert_close("T_hist", host(buf.T_hist), seq["T_hist"], FP64_TOL)
    assert_close("theta", host(buf.U_th), U_th, FP64_TOL)
    assert_close("U_T", host(buf.U_T), U_T, FP64_TOL)
    assert_close("Theta", host(Theta), [seq["Theta"]], FP64_TOL)
    assert_close("lambda", host(buf.V_l), V_l, FP64_TOL)
    assert_close("g", host(buf.V_g), V_g, FP64_TOL)
    assert_close("grad", host(grad), seq["grad"], FP64_TOL)
    st = op.stats()
    assert st["status"] == 0, st


def _oneshot_compare(name, precision, tol_t, tol_g, **solve_kw):
    prob, rho = case_problem(name)
    rho_old = W.rho_warm_perturb(rho, seed=1000, amp=0.05)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    op = gpu_operator(prob, precision, **solve_kw)
    buf = PassBuffers(op)
    buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
    buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
    op.assemble(dev(rho))
    Theta, grad = oneshot_pass(op, buf)
    torch.cuda.synchronize()
    assert_close("F_T", host(buf.F_T), ref["F_pri"][0], tol_t)
    assert_close("F_theta", host(buf.F_th), ref["F_pri"][1], tol_t)
    assert_close("G_T", host(buf.G_T), ref["G_pri_old"][0], tol_t)
    assert_close("G_theta", host(buf.G_th), ref["G_pri_old"][1], tol_t)
    assert_close("U_new", host(buf.U_T_new), ref["U"][0], tol_t)
    assert_close("theta_new", host(buf.U_th_new), ref["U"][1], tol_t)
    assert_close("T_hist", host(buf.T_hist), ref["T_hist"], tol_t)
    assert_close("Theta", host(Theta), [ref["Theta"]], tol_t)
    assert_close("F_lam", host(buf.F_l), ref["F_adj"][0], tol_g)
    assert_close("F_g", host(buf.F_g), ref["F_adj"][1], tol_g)
    assert_close("G_lam", host(buf.G_l), ref["G_adj_old"][0], tol_g)
    assert_close("G_g", host(buf.G_g), ref["G_adj_old"][1], tol_g)
    assert_close("V_lam", host(buf.V_l_new), ref["V"][0], tol_g)
    assert_close("V_g", host(buf.V_g_new), ref["V"][1], tol_g)
    assert_close("grad", host(grad), ref["grad"], tol_g)
    st = op.stats()
    assert st["status"] == 0, st
    return op, buf


@pytest.mark.parametrize("name", CASES)
def test_oneshot_pass_fp64(name):
    """Iteration body of Alg. 3 from a warm start of a nearby design: every intermediate of a2-a6."""
    _oneshot_compare(name, "fp64", FP64_TOL, FP64_TOL)


@pytest.mark.parametrize("precision", ["fp32_refine", "fp32_refine_all"])
@pytest.mark.parametrize("name", ["ragged_table1", "plain32", "paper_p20", "m1"])
def test_oneshot_pass_fp32_refine(name, precision):
    """FP32 CG with FP64 residual refinement for the fine-step solves (and, with
    fp32_refine_all, for the coarse-step solves too), against the FP64 oracle."""
    _oneshot_compare(name, precision, MIXED_T_TOL, MIXED_G_TOL, rtol=1e-10)


@pytest.mark.parametrize("name", ["ragged_table1", "paper_p20"])
def test_parareal_with_Ntau_iterations_is_sequential(name):
    """Sec. 4.2: N_tau Parareal iterations composed from the entry points reproduce the
    sequential solution (compared with the oracle's k-iteration Parareal and sequential pass)."""
    prob, rho = case_problem(name)
    oop = OracleOp(prob, rho)
    seq = o_sequential(oop)
    op = gpu_operator(prob)
    buf = PassBuffers(op)
    op.assemble(dev(rho))
    # coarse initial guess u^0 (Sec. 5.2): G sweep from u_0 with F = G (parareal_correct with F - G = 0)
    buf.U_T.zero_(); buf.U_th.zero_()
    zeros_T, zeros_th = op.zeros(op.Ntau, op.Nn), op.zeros(op.Ntau)
    op.parareal_correct(PTG_PRIMAL, zeros_T, zeros_th, zeros_T, zeros_th, buf.U_T, buf.U_th, T_hist=buf.T_hist)
    for _ in range(op.Ntau):
        op.fine_propagate_slices(buf.U_T, buf.U_th, buf.F_T, buf.F_th, T_hist=buf.T_hist)
        op.coarse_sweep(PTG_PRIMAL, buf.U_T, buf.U_th, buf.G_T, buf.G_th)
        buf.U_T_new[0].copy_(buf.U_T[0]); buf.U_th_new[0].copy_(buf.U_th[0])
        op.parareal_correct(PTG_PRIMAL, buf.F_T, buf.F_th, buf.G_T, buf.G_th, buf.U_T_new, buf.U_th_new,
                            T_hist=buf.T_hist)
        buf.U_T, buf.U_T_new = buf.U_T_new, buf.U_T
        buf.U_th, buf.U_th_new = buf.U_th_new, buf.U_th
    Theta = buf.U_th[op.Ntau:op.Ntau + 1]
    zl, zg = op.zeros(op.Ntau, op.Nn), op.zeros(op.Ntau, op.Ne)
    op.parareal_correct(PTG_ADJOINT, zl, zg, zl, zg, buf.V_l, buf.V_g, T_hist=buf.T_hist, Theta=Theta)
    for _ in range(op.Ntau):
        op.adjoint_sweep(buf.T_hist, Theta, buf.V_l, buf.V_g, buf.F_l, buf.F_g)
        op.coarse_sweep(PTG_ADJOINT, buf.V_l, buf.V_g, buf.G_l, buf.G_g, T_hist=buf.T_hist, Theta=Theta)
        op.parareal_correct(PTG_ADJOINT, buf.F_l, buf.F_g, buf.G_l, buf.G_g, buf.V_l_new, buf.V_g_new,
                            T_hist=buf.T_hist, Theta=Theta)
        buf.V_l, buf.V_l_new = buf.V_l_new, buf.V_l
        buf.V_g, buf.V_g_new = buf.V_g_new, buf.V_g
    par = o_parareal(oop, op.Ntau)
    assert_close("T_hist vs oracle parareal", host(buf.T_hist), par["T_hist"], FP64_TOL)
    assert_close("T_hist vs sequential", host(buf.T_hist), seq["T_hist"], FP64_TOL)
    assert_close("Theta", host(Theta), [seq["Theta"]], FP64_TOL)
    assert_close("grad", host(buf.V_g[0]), seq["grad"], FP64_TOL)


@pytest.mark.parametrize("name", ["ragged_table1", "plain32"])
def test_sensitivities_entry_point(name):
    """a6 on the oracle's sequential (lambda, T) histories reproduces the gradient (Eq. 4.7),
    both over the whole range and accumulated over two sub-ranges."""
    prob, rho = case_problem(name)
    seq = o_sequential(OracleOp(prob, rho))
    op = gpu_operator(prob)
    op.assemble(dev(rho))
    T = dev(seq["T_hist"])
    lam = dev(seq["lam"][1:prob.Nt + 1])
    grad = op.zeros(prob.Ne)
    op.sensitivities(lam, 1, prob.Nt, T, grad)
    assert_close("grad", host(grad), seq["grad"], FP64_TOL)
    g2 = op.zeros(prob.Ne)
    mid = prob.Nt // 3
    op.sensitivities(dev(seq["lam"][1:mid + 1]), 1, mid, T, g2)
    op.sensitivities(dev(seq["lam"][mid + 1:prob.Nt + 1]), mid + 1, prob.Nt, T[mid:], g2, hist_j0=mid)
    assert_close("grad (two ranges)", host(g2), seq["grad"], FP64_TOL)


def test_results_are_deterministic():
    """Fixed-order reductions: two identical passes agree bit for bit."""
    prob, rho = case_problem("ragged_table1")
    out = []
    for _ in range(2):
        op = gpu_operator(prob, "fp32_refine", rtol=1e-10)
        buf = PassBuffers(op)
        op.assemble(dev(rho))
        Theta, grad = sequential_pass(op, buf)
        out.append((host(buf.T_hist).copy(), host(grad).copy()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_design_out_of_range_is_reported():
    prob, rho = case_problem("tiny")
    op = gpu_operator(prob)
    bad = rho.copy()
    bad[2] = 1.5
    op.assemble(dev(bad))
    st = op.stats()
    assert st["status"] == -1 and st["fail_kind"] == 1
    bad[2] = np.nan
    op.reset_stats()
    op.assemble(dev(bad))
    assert op.stats()["status"] == -1


def test_iteration_limit_is_reported_not_hung():
    prob, rho = case_problem("ragged_table1")
    op = gpu_operator(prob, "fp64", cg_iters_max=1, refine_max=1)
    buf = PassBuffers(op)
    op.assemble(dev(rho))
    sequential_pass(op, buf)
    st = op.stats()
    assert st["status"] == -2 and st["fail_kind"] == 10 and st["fail_step"] == 1


def test_history_window_checked_on_host():
    prob, rho = case_problem("ragged_table1")
    op = gpu_operator(prob)
    buf = PassBuffers(op)
    op.assemble(dev(rho))
    with pytest.raises(PTGError):
        op.fine_propagate_slices(buf.U_T, buf.U_th, buf.F_T, buf.F_th, T_hist=buf.T_hist[:5])
    with pytest.raises(PTGError):
        op.adjoint_sweep(buf.T_hist[3:], buf.U_th[-1:], buf.V_l, buf.V_g, buf.F_l, buf.F_g, hist_j0=3)
