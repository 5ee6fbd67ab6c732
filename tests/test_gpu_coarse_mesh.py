"""Coarse propagators on the 2h mesh (the future work of Sec. 7.3) on the GPU against the oracle:
the one-shot pass element by element, its fixed point, Parareal's exactness after N_tau
iterations with this G, and the argument checks."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp
from oracle import coarse_states_from_sequential, oneshot_pass as o_oneshot, parareal as o_parareal
from oracle import sequential_pass as o_sequential
from oracle.coarse_mesh import CoarseMesh
from paper_2411_19030_gb300 import PassBuffers, PTGError, oneshot_pass, parareal_pass
from tests.gpu_helpers import FP64_TOL, MIXED_G_TOL, MIXED_T_TOL, assert_close, dev, ensure_built, gpu_operator, host
from tests.problems import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


CASES = {
    # ragged slabs, capacity SIMP (dC/drho != 0), the paper's time-varying load, a wide sink
    "table1": lambda: (make_problem(20, 16, Nt=32, Ntau=8, dt=1 / 32, material="table1", sink="left_wide",
                                    q_time=W.q_time_paper(32, 1 / 32)), W.rho_uniform(20, 16, 51, 0.05, 0.95)),
    # conductivity SIMP, the centred left sink, modified objective
    "modified": lambda: (make_problem(24, 20, Nt=24, Ntau=6, dt=1 / 24, modified_objective=True),
                         W.rho_uniform(24, 20, 52, 0.2, 0.8)),
    # the bottom sink of the paper's case, p = 20
    "paper": lambda: (make_problem(16, 16, Nt=40, Ntau=10, dt=1 / 40, material="table1", sink="bottom", p=20.0,
                                   q_time=W.q_time_paper(40, 1 / 40)), W.rho_branches(16, 16)),
}


def run(prob, rho, U_old, V_old, precision):
    op = gpu_operator(prob, precision, rtol=1e-13 if precision == "fp64" else 1e-10, coarse_mesh=True)
    buf = PassBuffers(op)
    buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
    buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
    op.assemble(dev(rho))
    Theta, grad = oneshot_pass(op, buf)
    torch.cuda.synchronize()
    return op, buf, Theta, grad


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine", "fp32_refine_all"])
@pytest.mark.parametrize("name", list(CASES))
def test_coarse_mesh_oneshot_pass_matches_oracle(name, precision):
    prob, rho = CASES[name]()
    rho_old = W.rho_warm_perturb(rho, seed=53, amp=0.05)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    oop = OracleOp(prob, rho)
    ref = o_oneshot(oop, U_old, V_old, coarse=CoarseMesh(oop))
    op, buf, Theta, grad = run(prob, rho, U_old, V_old, precision)
    tt, tg = (FP64_TOL, FP64_TOL) if precision == "fp64" else (MIXED_T_TOL, MIXED_G_TOL)
    assert_close("G_T", host(buf.G_T), ref["G_pri_old"][0], tt)
    assert_close("G_th", host(buf.G_th), ref["G_pri_old"][1], tt)
    assert_close("U_new", host(buf.U_T_new), ref["U"][0], tt)
    assert_close("theta_new", host(buf.U_th_new), ref["U"][1], tt)
    assert_close("T_hist", host(buf.T_hist), ref["T_hist"], tt)
    assert_close("Theta", host(Theta), [ref["Theta"]], tt)
    assert_close("G_lam", host(buf.G_l), ref["G_adj_old"][0], tg)
    assert_close("G_g", host(buf.G_g), ref["G_adj_old"][1], tg)
    assert_close("V_lam", host(buf.V_l_new), ref["V"][0], tg)
    assert_close("V_g", host(buf.V_g_new), ref["V"][1], tg)
    assert_close("grad", host(grad), ref["grad"], tg)
    assert op.stats()["status"] == 0


def test_coarse_mesh_fixed_point_on_gpu():
    """Warm-started from the exact sequential coarse states of the same design the pass returns
    the sequential result, whatever G is."""
    prob, rho = CASES["table1"]()
    seq = o_sequential(OracleOp(prob, rho))
    U, V, _ = coarse_states_from_sequential(OracleOp(prob, rho), seq)
    op, buf, Theta, grad = run(prob, rho, U, V, "fp64")
    assert_close("T_hist", host(buf.T_hist), seq["T_hist"], FP64_TOL)
    assert_close("Theta", host(Theta), [seq["Theta"]], FP64_TOL)
    assert_close("grad", host(grad), seq["grad"], FP64_TOL)


def test_coarse_mesh_parareal_matches_oracle_and_is_exact_after_Ntau_iterations():
    prob, rho = CASES["modified"]()
    oop = OracleOp(prob, rho)
    seq = o_sequential(oop)
    for k, ref in ((2, o_parareal(oop, 2, coarse=CoarseMesh(oop))), (prob.Ntau, seq)):
        op = gpu_operator(prob, "fp64", rtol=1e-13, coarse_mesh=True)
        buf = PassBuffers(op)
        op.assemble(dev(rho))
        Theta, grad = parareal_pass(op, buf, k)
        torch.cuda.synchronize()
        assert_close(f"T_hist k={k}", host(buf.T_hist), ref["T_hist"], FP64_TOL)
        assert_close(f"grad k={k}", host(grad), ref["grad"], FP64_TOL)


def test_coarse_mesh_needs_even_grids():
    prob = make_problem(13, 10, Nt=8, Ntau=4)
    with pytest.raises(PTGError):
        gpu_operator(prob, "fp64", coarse_mesh=True)
