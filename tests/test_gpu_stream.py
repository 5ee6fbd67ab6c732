"""The streamed fine propagators (ptg_solve.fine_stream = 2): every slice a group of CTAs of one
launch with its Krylov vectors in global memory, as used on large grids.  Forced on small
problems here: the one-shot pass must match the oracle (FP64 and mixed precision; capacity SIMP
and the modified objective; ragged grids), with one CTA per slice (as at 512 x 512) and with
several CTAs per slice whose reductions and neighbour rows go through global memory, and match
the on-chip path to the solver tolerance."""
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
    # few slices: many CTAs per slice (global-memory reductions and neighbour rows)
    "ragged_table1": lambda: (make_problem(26, 19, Nt=24, Ntau=4, dt=0.6 / 24, material="table1", sink="left_wide",
                                           q_time=W.q_time_paper(24, 0.6 / 24)), W.rho_uniform(26, 19, 81, 0.05, 0.95)),
    "modified_objective": lambda: (make_problem(30, 22, Nt=16, Ntau=8, dt=1 / 16, material="table1", sink="bottom",
                                                modified_objective=True), W.rho_uniform(30, 22, 82, 0.1, 0.9)),
    # more slices than SMs: one CTA per slice
    "one_cta_per_slice": lambda: (make_problem(9, 7, Nt=160, Ntau=160, dt=1 / 160, material="simp_k", sink="left_wide"),
                                  W.rho_uniform(9, 7, 83, 0.2, 0.8)),
}


def run(prob, rho, U_old, V_old, precision, stream, **kw):
    op = gpu_operator(prob, precision, rtol=1e-13 if precision == "fp64" else 1e-10, fine_stream=stream, **kw)
    buf = PassBuffers(op)
    buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
    buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
    op.assemble(dev(rho))
    Theta, grad = oneshot_pass(op, buf)
    torch.cuda.synchronize()
    return op, buf, Theta, grad


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("name", list(CASES))
def test_streamed_fine_propagators_match_oracle(name, precision):
    prob, rho = CASES[name]()
    rho_old = W.rho_warm_perturb(rho, seed=84, amp=0.05)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    op, buf, Theta, grad = run(prob, rho, U_old, V_old, precision, 2)
    assert op.plan(0, prob.Ntau)["nthreads"] == 512            # the streamed plan ran
    tol_t, tol_g = (FP64_TOL, FP64_TOL) if precision == "fp64" else (MIXED_T_TOL, MIXED_G_TOL)
    assert_close("F_T", host(buf.F_T), ref["F_pri"][0], tol_t)
    assert_close("F_theta", host(buf.F_th), ref["F_pri"][1], tol_t)
    assert_close("T_hist", host(buf.T_hist), ref["T_hist"], tol_t)
    assert_close("Theta", host(Theta), [ref["Theta"]], tol_t)
    assert_close("F_lam", host(buf.F_l), ref["F_adj"][0], tol_g)
    assert_close("F_g", host(buf.F_g), ref["F_adj"][1], tol_g)
    assert_close("grad", host(grad), ref["grad"], tol_g)
    st = op.stats()
    assert st["status"] == 0, st
    # the on-chip path gives the same pass to the solver tolerance
    _, buf2, Theta2, grad2 = run(prob, rho, U_old, V_old, precision, 1)
    assert_close("streamed vs on chip", host(grad), host(grad2), 1e-9 if precision == "fp64" else 1e-6)


def test_streamed_path_is_deterministic():
    prob, rho = CASES["ragged_table1"]()
    U, V, _ = coarse_states_from_sequential(OracleOp(prob, rho))
    a = run(prob, rho, U, V, "fp32_refine", 2)
    b = run(prob, rho, U, V, "fp32_refine", 2)
    assert np.array_equal(host(a[3]), host(b[3])) and np.array_equal(host(a[1].T_hist), host(b[1].T_hist))


def _plans(prob, stream):
    op = gpu_operator(prob, "fp32_refine", fine_stream=stream)
    return [op.plan(kind, prob.Ntau) for kind in (0, 3)]


def test_library_streams_only_where_no_cluster_holds_a_slice():
    # 512 x 512: slabs of a slice fit no 16-CTA cluster, so fine_stream 0 takes the streamed plan
    big = make_problem(512, 512, Nt=16, Ntau=8, dt=1 / 16, material="table1", sink="left_wide")
    auto, forced = _plans(big, 0), _plans(big, 2)
    assert auto == forced and all(p["nthreads"] == 512 for p in auto)
    # 128 x 128: clusters hold a slice and the on-chip plan stays
    small = make_problem(128, 128, Nt=16, Ntau=8, dt=1 / 16, material="table1", sink="left_wide")
    assert _plans(small, 0) == _plans(small, 1)


MG_CASES = {
    # three levels (40 x 32 -> 20 x 16 -> 10 x 8), several CTAs per slice
    "table1_40x32": lambda: (make_problem(40, 32, Nt=24, Ntau=4, dt=0.6 / 24, material="table1", sink="left_wide",
                                          q_time=W.q_time_paper(24, 0.6 / 24)), W.rho_uniform(40, 32, 85, 0.05, 0.95)),
    # two levels, one CTA per slice
    "one_cta_16": lambda: (make_problem(16, 16, Nt=160, Ntau=160, dt=1 / 160, material="simp_k", sink="left_wide"),
                           W.rho_uniform(16, 16, 86, 0.2, 0.8)),
}


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("name", list(MG_CASES))
def test_streamed_fine_propagators_with_multigrid_match_oracle(name, precision):
    """local_steps = 3: the streamed fine CG preconditioned by the multigrid V-cycle of C/dt + K."""
    prob, rho = MG_CASES[name]()
    rho_old = W.rho_warm_perturb(rho, seed=87, amp=0.05)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    its = {}
    for ls in (3, 1):
        op, buf, Theta, grad = run(prob, rho, U_old, V_old, precision, 2, local_steps=ls)
        tol_t, tol_g = (FP64_TOL, FP64_TOL) if precision == "fp64" else (MIXED_T_TOL, MIXED_G_TOL)
        assert_close(f"F_T[{ls}]", host(buf.F_T), ref["F_pri"][0], tol_t)
        assert_close(f"T_hist[{ls}]", host(buf.T_hist), ref["T_hist"], tol_t)
        assert_close(f"F_lam[{ls}]", host(buf.F_l), ref["F_adj"][0], tol_g)
        assert_close(f"F_g[{ls}]", host(buf.F_g), ref["F_adj"][1], tol_g)
        assert_close(f"grad[{ls}]", host(grad), ref["grad"], tol_g)
        st = op.stats()
        assert st["status"] == 0, st
        its[ls] = st["kind_cg_iters"][0] / st["kind_solves"][0]
    assert its[3] < its[1], its                  # the cycle cuts the fine-step iterations
