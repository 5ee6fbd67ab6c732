"""The adjoint coarse propagator as two Theta-free parts (ptg_coarse_adjoint_split) combined with
the source scale of Eq. 4.6 once Theta is known (ptg_coarse_adjoint_combine), and the one-shot
pass that runs those parts on a second stream beside the forward correction sweep.

G_adj is affine in the adjoint source scale c (Eq. 4.6: c = Theta^(1-p)/Ne; p/Ne for the
modified objective of Sec. 7.1), so H + c S must equal the direct G_adj to the solver
tolerance, and the overlapped pass must match the oracle's one-shot pass like the plain one."""
from __future__ import annotations

import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp
from oracle import coarse_states_from_sequential, oneshot_pass as o_oneshot
from paper_2411_19030_gb300 import PTG_ADJOINT, PassBuffers, oneshot_pass
from tests.gpu_helpers import (FP64_TOL, MIXED_G_TOL, MIXED_T_TOL, assert_close, dev, ensure_built, gpu_operator,
                               host)
from tests.problems import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _problem(modified=False):
    Nt, Ntau = 30, 6
    prob = make_problem(26, 19, Nt=Nt, Ntau=Ntau, dt=0.6 / Nt, material="table1", sink="left_wide",
                        q_time=W.q_time_paper(Nt, 0.6 / Nt), modified_objective=modified)
    rho = W.rho_uniform(26, 19, 61, 0.05, 0.95)
    return prob, rho, W.rho_warm_perturb(rho, seed=62, amp=0.05)


@pytest.mark.parametrize("modified", [False, True])
def test_split_parts_combine_to_the_direct_coarse_adjoint(modified):
    prob, rho, rho_old = _problem(modified)
    U_old, V_old, seq = coarse_states_from_sequential(OracleOp(prob, rho_old))
    op = gpu_operator(prob, "fp64", rtol=1e-13)
    op.assemble(dev(rho))
    T_hist, V_l, V_g = dev(seq["T_hist"]), dev(V_old[0]), dev(V_old[1])
    Theta = dev([seq["Theta"] * 1.01])
    G_l, G_g = op.zeros(prob.Ntau, prob.Nn), op.zeros(prob.Ntau, prob.Ne)
    op.coarse_sweep(PTG_ADJOINT, V_l, V_g, G_l, G_g, T_hist=T_hist, Theta=Theta)
    H_l, H_g, S_l, S_g = (torch.zeros_like(t) for t in (G_l, G_g, G_l, G_g))
    C_l, C_g = torch.zeros_like(G_l), torch.zeros_like(G_g)
    # two halves of the slice range, as two processes would split it
    for s0, ns in ((0, 2), (2, 4)):
        op.coarse_adjoint_split(V_l, V_g, T_hist, H_l, H_g, S_l, S_g, s0=s0, ns=ns)
        op.coarse_adjoint_combine(Theta, H_l, H_g, S_l, S_g, C_l, C_g, s0=s0, ns=ns)
    torch.cuda.synchronize()
    assert_close("lambda", host(C_l), host(G_l), 1e-11)
    assert_close("g", host(C_g), host(G_g), 1e-11)
    assert op.stats()["status"] == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_overlapped_pass_matches_oracle_and_plain_order(precision):
    prob, rho, rho_old = _problem()
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    op = gpu_operator(prob, precision, rtol=1e-13 if precision == "fp64" else 1e-10)
    assert op.can_overlap_adjoint_coarse()
    out = {}
    for overlap in (True, False):
        buf = PassBuffers(op)
        buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
        buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
        op.assemble(dev(rho))
        Theta, grad = oneshot_pass(op, buf, overlap=overlap)
        torch.cuda.synchronize()
        tol_t, tol_g = (FP64_TOL, FP64_TOL) if precision == "fp64" else (MIXED_T_TOL, MIXED_G_TOL)
        assert_close(f"T_hist[{overlap}]", host(buf.T_hist), ref["T_hist"], tol_t)
        assert_close(f"Theta[{overlap}]", host(Theta), [ref["Theta"]], tol_t)
        assert_close(f"G_lam[{overlap}]", host(buf.G_l), ref["G_adj_old"][0], tol_g)
        assert_close(f"V_new[{overlap}]", host(buf.V_l_new), ref["V"][0], tol_g)
        assert_close(f"grad[{overlap}]", host(grad), ref["grad"], tol_g)
        out[overlap] = host(grad).copy()
    assert_close("overlapped vs plain order", out[True], out[False], 1e-9 if precision == "fp64" else 1e-6)
    assert op.stats()["status"] == 0


def test_overlap_is_off_where_it_does_not_apply():
    # M = 1: the rows G_adj reads are the rows the forward sweep corrects
    prob = make_problem(12, 10, Nt=6, Ntau=6, dt=0.1, material="table1", sink="left_wide")
    assert not gpu_operator(prob, "fp64").can_overlap_adjoint_coarse()
    prob = make_problem(12, 10, Nt=12, Ntau=6, dt=0.1, material="table1", sink="left_wide")
    assert gpu_operator(prob, "fp64").can_overlap_adjoint_coarse()
    assert not gpu_operator(prob, "fp64", coarse_mesh=True).can_overlap_adjoint_coarse()


def test_overlap_is_off_for_cooperative_grid_plans():
    # grid_wide = 2 plans every kind as groups of a cooperative launch, which share the op's
    # grid workspace: the parts must not run beside the forward sweep
    prob = make_problem(12, 10, Nt=12, Ntau=6, dt=0.1, material="table1", sink="left_wide")
    assert not gpu_operator(prob, "fp64", grid_wide=2).can_overlap_adjoint_coarse()
