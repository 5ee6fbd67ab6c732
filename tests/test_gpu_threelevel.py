"""The three-level cycle of the coarse-step solves (ptg_solve.twolevel = PTG_TWOLEVEL_THREELEVEL):
the two-grid cycle whose coarse correction is itself a two-grid cycle on the 2h level (bilinear
P1 from the nodes (2I, 2J), Galerkin A1 = P1^T A P1, slab-local damped-Jacobi smoothing on the
2h rows of each CTA) over aggregates of 2h nodes with a dense inverse.  It changes only how
many CG iterations a coarse-step solve takes: the one-shot pass must match the oracle for every
cluster size and precision, need fewer coarse and correction CG iterations than the two-grid
cycle, and fall back to the two-grid cycle where it does not apply (odd grids)."""
from __future__ import annotations

import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp
from oracle import coarse_states_from_sequential, oneshot_pass as o_oneshot
from paper_2411_19030_gb300 import PassBuffers, oneshot_pass
from tests.gpu_helpers import FP64_TOL, MIXED_G_TOL, MIXED_T_TOL, assert_close, dev, ensure_built, gpu_operator, host
from tests.problems import make_problem

pytestmark = pytest.mark.gpu

COARSE_KINDS = (1, 2, 4, 5)
COARSE_NAMES = ("coarse_primal", "correct_primal", "coarse_adjoint", "correct_adjoint")


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _case(nx, ny, Nt, Ntau, material="simp_k", sink="left", seed=21):
    prob = make_problem(nx, ny, Nt=Nt, Ntau=Ntau, dt=1 / Nt, material=material, sink=sink,
                        q_time=W.q_time_paper(Nt, 1 / Nt) if material == "table1" else None)
    rho = W.rho_uniform(nx, ny, seed, 0.05, 0.95)
    rho_old = W.rho_warm_perturb(rho, seed=seed + 1, amp=0.05)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    return prob, rho, U_old, V_old, ref


@pytest.fixture(scope="module")
def case():
    """64 x 48 elements: a 33 x 25 2h level, 8 slices of 8 steps, warm start of a nearby design."""
    return _case(64, 48, 64, 8)


def run_pass(case, twolevel, cs=0, precision="fp32_refine", smooth=0):
    prob, rho, U_old, V_old, _ = case
    op = gpu_operator(prob, precision, rtol=1e-13 if precision == "fp64" else 1e-10, twolevel=twolevel,
                      smooth_steps=smooth)
    if cs:
        for kind in COARSE_KINDS:
            op.set_plan(kind, cs, 1 if cs >= 8 else 2)
    buf = PassBuffers(op)
    buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
    buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
    op.assemble(dev(rho))
    Theta, grad = oneshot_pass(op, buf)
    torch.cuda.synchronize()
    return op, buf, Theta, grad


def check(case, op, buf, Theta, grad, tol_t=MIXED_T_TOL, tol_g=MIXED_G_TOL):
    ref = case[4]
    assert_close("G_T", host(buf.G_T), ref["G_pri_old"][0], tol_t)
    assert_close("U_new", host(buf.U_T_new), ref["U"][0], tol_t)
    assert_close("T_hist", host(buf.T_hist), ref["T_hist"], tol_t)
    assert_close("Theta", host(Theta), [ref["Theta"]], tol_t)
    assert_close("G_lam", host(buf.G_l), ref["G_adj_old"][0], tol_g)
    assert_close("V_lam", host(buf.V_l_new), ref["V"][0], tol_g)
    assert_close("grad", host(grad), ref["grad"], tol_g)
    assert op.stats()["status"] == 0


@pytest.mark.parametrize("precision", ["fp32_refine", "fp32_refine_all"])
@pytest.mark.parametrize("cs", [2, 4, 8, 16])
def test_threelevel_pass_matches_oracle_for_every_cluster_size(case, cs, precision):
    op, buf, Theta, grad = run_pass(case, "threelevel", cs, precision)
    assert op.plan(1, 1)["cs"] == cs
    check(case, op, buf, Theta, grad)


def test_threelevel_fp64_path_keeps_the_fp64_tolerance(case):
    op, buf, Theta, grad = run_pass(case, "threelevel", 0, "fp64")
    check(case, op, buf, Theta, grad, FP64_TOL, FP64_TOL)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine_all"])
def test_threelevel_needs_fewer_iterations_than_the_two_grid_cycle(case, precision):
    runs = {m: run_pass(case, m, 0, precision) for m in ("threelevel", "vcycle")}
    tol = (FP64_TOL, FP64_TOL) if precision == "fp64" else (MIXED_T_TOL, MIXED_G_TOL)
    for m in runs:
        check(case, *runs[m], *tol)
    k = {m: runs[m][0].stats()["by_kind"] for m in runs}
    for name in COARSE_NAMES:
        assert k["threelevel"][name]["solves"] == k["vcycle"][name]["solves"] > 0
        assert k["threelevel"][name]["cg_iters"] < 0.8 * k["vcycle"][name]["cg_iters"], (name, k)


@pytest.mark.parametrize("nx,ny", [(26, 19), (13, 9)])
def test_threelevel_falls_back_on_odd_grids(nx, ny):
    case = _case(nx, ny, 24, 4, material="table1", sink="left_wide", seed=31)
    out = {}
    for m in ("threelevel", "vcycle"):
        # the same smoothing steps for both (the three-level default is 3, the two-grid cycle's 4)
        op, buf, Theta, grad = run_pass(case, m, 0, "fp64", smooth=3)
        check(case, op, buf, Theta, grad, FP64_TOL, FP64_TOL)
        out[m] = host(grad)
    # the same two-grid cycle runs either way
    assert (out["threelevel"] == out["vcycle"]).all()


@pytest.mark.parametrize("design", ["branches_table1_bottom", "uniform_simp_left"])
def test_threelevel_on_high_contrast_designs(design):
    from paper_2411_19030_gb300 import parareal_pass
    n, Nt = 64, 256
    if design == "branches_table1_bottom":
        prob, rho = make_problem(n, Nt=Nt, Ntau=16, dt=1 / Nt, material="table1", sink="bottom"), W.rho_branches(n, n)
    else:
        prob, rho = make_problem(n, Nt=Nt, Ntau=16, dt=1 / Nt), W.rho_uniform(n, n, 1, 0.2, 0.8)
    its = {}
    for tl in ("threelevel", "vcycle"):
        op = gpu_operator(prob, "fp64", rtol=1e-10, twolevel=tl)
        buf = PassBuffers(op)
        op.assemble(dev(rho))
        parareal_pass(op, buf, 1)
        torch.cuda.synchronize()
        assert op.stats()["status"] == 0
        st = op.stats()["by_kind"]["correct_primal"]
        its[tl] = st["cg_iters"] / st["solves"]
    assert its["threelevel"] < 0.8 * its["vcycle"], its
