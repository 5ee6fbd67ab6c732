"""Initial guesses of the time-step solves (ptg_solve.initial_guess): starting each fine CG from
the polynomial extrapolation through the last n states of its run and each batched coarse CG
from the guess state at the other end of its slice changes only where the iterations start, so
the one-shot pass and the sequential pass match the oracle with every setting, and the
extrapolated start takes fewer fine CG iterations (the coarse-step guess helps as far as the
guess state is close to G of its predecessor, which a warm start from another design is not
always: there it must not cost iterations)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp
from oracle import coarse_states_from_sequential, oneshot_pass as o_oneshot, sequential_pass as o_sequential
from paper_2411_19030_gb300 import PassBuffers, oneshot_pass, sequential_pass
from tests.gpu_helpers import FP64_TOL, MIXED_G_TOL, MIXED_T_TOL, assert_close, dev, ensure_built, gpu_operator, host
from tests.problems import make_problem

pytestmark = pytest.mark.gpu

FINE = ("fine_primal", "fine_adjoint")
COARSE = ("coarse_primal", "coarse_adjoint", "correct_primal", "correct_adjoint")


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.fixture(scope="module")
def case():
    """48 x 40 elements (ragged slabs), the paper's time-varying load, 96 steps in 8 slices, warm
    start from a nearby design."""
    prob = make_problem(48, 40, Nt=96, Ntau=8, dt=1 / 96, material="table1", sink="left_wide",
                        q_time=W.q_time_paper(96, 1 / 96))
    rho = W.rho_uniform(48, 40, 71, 0.05, 0.95)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, W.rho_warm_perturb(rho, seed=72, amp=0.05)))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    return prob, rho, U_old, V_old, ref


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_oneshot_pass_with_either_initial_guess_matches_oracle(case, precision):
    prob, rho, U_old, V_old, ref = case
    tt, tg = (FP64_TOL, FP64_TOL) if precision == "fp64" else (MIXED_T_TOL, MIXED_G_TOL)
    its = {}
    for guess in (1, 2, 3, 4):
        # rtol 1e-12 in FP64: with the FP32 two-grid preconditioner the FP64 CG of the coarse
        # steps of this case stalls just above 1e-13 whatever its start
        op = gpu_operator(prob, precision, rtol=1e-12 if precision == "fp64" else 1e-10, initial_guess=guess)
        buf = PassBuffers(op)
        buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
        buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
        op.assemble(dev(rho))
        Theta, grad = oneshot_pass(op, buf)
        torch.cuda.synchronize()
        assert_close(f"T_hist {guess}", host(buf.T_hist), ref["T_hist"], tt)
        assert_close(f"G_T {guess}", host(buf.G_T), ref["G_pri_old"][0], tt)
        assert_close(f"U_new {guess}", host(buf.U_T_new), ref["U"][0], tt)
        assert_close(f"Theta {guess}", host(Theta), [ref["Theta"]], tt)
        assert_close(f"G_lam {guess}", host(buf.G_l), ref["G_adj_old"][0], tg)
        assert_close(f"V_lam {guess}", host(buf.V_l_new), ref["V"][0], tg)
        assert_close(f"grad {guess}", host(grad), ref["grad"], tg)
        st = op.stats()
        assert st["status"] == 0, st
        its[guess] = {k: st["by_kind"][k]["cg_iters"] for k in FINE + COARSE}
    for k in FINE:
        assert its[4][k] < its[2][k] < its[1][k], (k, its)
    for k in COARSE:
        assert its[4][k] <= its[1][k], (k, its)


def test_sequential_pass_with_extrapolated_start_matches_oracle():
    """Chained runs over a smooth solution (4 slices of 64 steps, each slice extrapolating from
    its own start), where the cubic start saves most of the fine CG iterations."""
    prob = make_problem(32, 24, Nt=256, Ntau=4, dt=1 / 256)
    rho = W.rho_uniform(32, 24, 73, 0.2, 0.8)
    oop = OracleOp(prob, rho)
    seq = o_sequential(oop)
    (U_T, _), (V_l, V_g), _ = coarse_states_from_sequential(oop, seq)
    its = {}
    for guess in (1, 4):
        op = gpu_operator(prob, "fp64", rtol=1e-13, initial_guess=guess)
        buf = PassBuffers(op)
        op.assemble(dev(rho))
        Theta, grad = sequential_pass(op, buf)
        assert_close(f"T_hist {guess}", host(buf.T_hist), seq["T_hist"], FP64_TOL)
        assert_close(f"U_T {guess}", host(buf.U_T), U_T, FP64_TOL)
        assert_close(f"lambda {guess}", host(buf.V_l), V_l, FP64_TOL)
        assert_close(f"g {guess}", host(buf.V_g), V_g, FP64_TOL)
        assert_close(f"grad {guess}", host(grad), seq["grad"], FP64_TOL)
        st = op.stats()
        assert st["status"] == 0, st
        its[guess] = {k: st["by_kind"][k]["cg_iters"] for k in FINE}
    for k in FINE:
        assert its[4][k] < 0.7 * its[1][k], (k, its)


def test_slice_recomputed_alone_repeats_the_chained_run_bit_for_bit():
    """Checkpointed differentiation recomputes a slice from its start state alone; the initial
    guesses restart at every slice start, so the recomputed history equals the chained run's,
    bit for bit, and a chained run without a history window ends in the same states."""
    from paper_2411_19030_gb300 import PTG_SLICES_CHAINED, PTG_SLICES_PARALLEL
    prob = make_problem(32, 24, Nt=128, Ntau=4, dt=1 / 128)
    rho = W.rho_uniform(32, 24, 74, 0.2, 0.8)
    op = gpu_operator(prob, "fp64", rtol=1e-13)
    buf = PassBuffers(op)
    op.assemble(dev(rho))
    sequential_pass(op, buf)
    T_full = host(buf.T_hist).copy()
    U_full = host(buf.U_T).copy()
    M = prob.M
    window = torch.zeros((M + 1, prob.Nn), dtype=torch.float64, device="cuda")
    for s in range(prob.Ntau):
        window.zero_()
        op.fine_propagate_slices(buf.U_T, buf.U_th, buf.F_T, buf.F_th, T_hist=window, hist_j0=M * s,
                                 schedule=PTG_SLICES_PARALLEL, s0=s, ns=1)
        assert np.array_equal(host(window)[1:], T_full[M * s + 1:M * (s + 1) + 1]), s
    U2 = torch.zeros_like(buf.U_T)
    th2 = torch.zeros_like(buf.U_th)
    U2[0].copy_(buf.U_T[0])
    th2[0].copy_(buf.U_th[0])
    op.fine_propagate_slices(U2, th2, U2[1:], th2[1:], T_hist=None, schedule=PTG_SLICES_CHAINED)
    assert np.array_equal(host(U2), U_full)
    assert op.stats()["status"] == 0


def test_initial_guess_out_of_range_is_rejected():
    from paper_2411_19030_gb300 import PTGError
    prob = make_problem(8, 8, Nt=4, Ntau=2)
    with pytest.raises(PTGError):
        gpu_operator(prob, "fp64", initial_guess=5)
