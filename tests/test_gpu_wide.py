"""Single FP64 systems over a cooperative grid (one CTA per SM at most, global-memory halos and
reductions behind a counting grid barrier) against the oracle and against the one-cluster
path: the sequential pass (chained fine kinds) and the correction sweeps of the one-shot
pass."""
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


CASES = {
    "square64": lambda: (make_problem(64, Nt=64, Ntau=8, dt=1 / 64), W.rho_uniform(64, 64, 2, 0.05, 0.95)),
    "ragged_table1": lambda: (make_problem(13, 9, Nt=24, Ntau=4, dt=1 / 24, material="table1", sink="left_wide",
                                           q_time=W.q_time_paper(24, 1 / 24)), W.rho_uniform(13, 9, 3, 0.05, 0.95)),
    "tall": lambda: (make_problem(20, 96, Nt=30, Ntau=5, dt=1e-3, material="table1", sink="bottom", p=20.0),
                     W.rho_uniform(20, 96, 4, 0.1, 0.9)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_wide_sequential_pass_matches_oracle_and_cluster_path(name):
    prob, rho = CASES[name]()
    seq = o_sequential(OracleOp(prob, rho))
    out = {}
    for wide in (True, False):
        op = gpu_operator(prob, "fp64", grid_wide=2 if wide else 0)
        if wide:
            assert op.plan(0, 1)["cs"] > 16 or prob.ny < 34
        buf = PassBuffers(op)
        op.assemble(dev(rho))
        Theta, grad = sequential_pass(op, buf)
        torch.cuda.synchronize()
        assert_close(f"T_hist[{wide}]", host(buf.T_hist), seq["T_hist"], FP64_TOL)
        assert_close(f"Theta[{wide}]", host(Theta), [seq["Theta"]], FP64_TOL)
        assert_close(f"grad[{wide}]", host(grad), seq["grad"], FP64_TOL)
        assert op.stats()["status"] == 0, op.stats()
        out[wide] = host(grad).copy()
    assert_close("wide vs cluster", out[True], out[False], 1e-11)


@pytest.mark.parametrize("mode", ["additive", "vcycle1", "vcycle3"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("name", ["square64", "tall"])
def test_wide_correction_sweeps_match_oracle(name, precision, mode):
    prob, rho = CASES[name]()
    rho_old = W.rho_warm_perturb(rho, seed=41, amp=0.05)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    tol_t, tol_g = (FP64_TOL, FP64_TOL) if precision == "fp64" else (MIXED_T_TOL, MIXED_G_TOL)
    op = gpu_operator(prob, precision, rtol=1e-13 if precision == "fp64" else 1e-10, grid_wide=2,
                      twolevel=mode[:6] if mode.startswith("vcycle") else mode,
                      smooth_steps=int(mode[6:]) if mode.startswith("vcycle") else 0)
    assert op.plan(2, 1)["cs"] > 16
    buf = PassBuffers(op)
    buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
    buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
    op.assemble(dev(rho))
    Theta, grad = oneshot_pass(op, buf)
    torch.cuda.synchronize()
    assert_close("U_new", host(buf.U_T_new), ref["U"][0], tol_t)
    assert_close("T_hist", host(buf.T_hist), ref["T_hist"], tol_t)
    assert_close("Theta", host(Theta), [ref["Theta"]], tol_t)
    assert_close("V_lam", host(buf.V_l_new), ref["V"][0], tol_g)
    assert_close("grad", host(grad), ref["grad"], tol_g)
    assert op.stats()["status"] == 0, op.stats()


def test_wide_path_is_deterministic():
    prob, rho = CASES["square64"]()
    op = gpu_operator(prob, "fp64", grid_wide=2)
    buf = PassBuffers(op)
    op.assemble(dev(rho))
    runs = []
    for _ in range(2):
        Theta, grad = sequential_pass(op, buf)
        torch.cuda.synchronize()
        runs.append((host(Theta).copy(), host(grad).copy()))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("mode", ["additive", "vcycle1", "vcycle3"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("name", ["square64", "ragged_table1", "tall"])
def test_grouped_launches_for_every_kind_match_oracle(name, precision, mode):
    """grid_wide = 2: every kind in groups of CTAs of one cooperative launch (several slices
    per launch, one group each), the one-shot pass against the oracle."""
    prob, rho = CASES[name]()
    rho_old = W.rho_warm_perturb(rho, seed=43, amp=0.05)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    tol_t, tol_g = (FP64_TOL, FP64_TOL) if precision == "fp64" else (MIXED_T_TOL, MIXED_G_TOL)
    op = gpu_operator(prob, precision, rtol=1e-13 if precision == "fp64" else 1e-10, grid_wide=2,
                      twolevel=mode[:6] if mode.startswith("vcycle") else mode,
                      smooth_steps=int(mode[6:]) if mode.startswith("vcycle") else 0)
    buf = PassBuffers(op)
    buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
    buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
    op.assemble(dev(rho))
    Theta, grad = oneshot_pass(op, buf)
    torch.cuda.synchronize()
    assert_close("F_T", host(buf.F_T), ref["F_pri"][0], tol_t)
    assert_close("G_T", host(buf.G_T), ref["G_pri_old"][0], tol_t)
    assert_close("T_hist", host(buf.T_hist), ref["T_hist"], tol_t)
    assert_close("Theta", host(Theta), [ref["Theta"]], tol_t)
    assert_close("F_lam", host(buf.F_l), ref["F_adj"][0], tol_g)
    assert_close("grad", host(grad), ref["grad"], tol_g)
    assert op.stats()["status"] == 0, op.stats()


def test_512_grid_runs_in_groups_fixed_point_and_symmetry():
    """512 x 512 (no slab fits a 16-CTA cluster): a short time grid.  Warm started from the
    exact sequential coarse states of the same design, the one-shot pass returns the
    sequential result; the uniform design with the centred sink gives a gradient symmetric
    about mid-height."""
    prob = make_problem(512, Nt=64, Ntau=4, dt=1 / 4096)
    rho = np.full(prob.Ne, 0.4)
    seq_op = gpu_operator(prob, "fp64", rtol=1e-13)
    assert seq_op.plan(0, 4)["cs"] > 16
    sbuf = PassBuffers(seq_op)
    seq_op.assemble(dev(rho))
    Th_s, g_s = sequential_pass(seq_op, sbuf)
    op = gpu_operator(prob, "fp32_refine", rtol=1e-10)
    buf = PassBuffers(op)
    for a, b in ((buf.U_T, sbuf.U_T), (buf.U_th, sbuf.U_th), (buf.V_l, sbuf.V_l), (buf.V_g, sbuf.V_g)):
        a.copy_(b)
    op.assemble(dev(rho))
    Theta, grad = oneshot_pass(op, buf)
    torch.cuda.synchronize()
    assert seq_op.stats()["status"] == 0 and op.stats()["status"] == 0
    assert_close("Theta", host(Theta), host(Th_s), MIXED_T_TOL)
    assert_close("grad", host(grad), host(g_s), MIXED_G_TOL)
    g = host(g_s).reshape(512, 512)
    assert_close("mirror", g[::-1, :], g, 1e-9)
