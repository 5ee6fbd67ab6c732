"""Two-level preconditioners of the coarse-step solves (aggregation coarse space), additive
(D^-1 + P Ac^-1 P^T) and the symmetric V(1,1) two-grid cycle with damped-Jacobi smoothing: the
one-shot pass with either matches the oracle for every cluster size (the restricted residual is
summed across the CTAs of a cluster whose slabs split aggregate rows differently; the V-cycle
also smooths across slab edges), and they need fewer CG iterations than Jacobi alone on the
coarse and correction solves, the V-cycle fewer than the additive form."""
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

COARSE_KINDS = (1, 2, 4, 5)   # coarse_primal, correct_primal, coarse_adjoint, correct_adjoint


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.fixture(scope="module")
def case():
    """64 x 48 elements (16 x 12 aggregates of 4 x 4 nodes, the last ones larger), 64 steps in
    8 slices, warm start of a nearby design."""
    prob = make_problem(64, 48, Nt=64, Ntau=8, dt=1 / 64)
    rho = W.rho_uniform(64, 48, 11, 0.05, 0.95)
    rho_old = W.rho_warm_perturb(rho, seed=12, amp=0.05)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    return prob, rho, U_old, V_old, ref


def run_pass(case, twolevel, cs=0, precision="fp32_refine"):
    """twolevel: "none", "additive", "vcycle" or "vcycle<k>" (k smoothing steps)."""
    prob, rho, U_old, V_old, _ = case
    smooth = int(twolevel[6:]) if twolevel.startswith("vcycle") and len(twolevel) > 6 else 0
    op = gpu_operator(prob, precision, rtol=1e-13 if precision == "fp64" else 1e-10,
                      twolevel=twolevel[:6] if smooth else twolevel, smooth_steps=smooth)
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


MODES = ["additive", "vcycle1", "vcycle3"]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("precision", ["fp32_refine", "fp32_refine_all"])
@pytest.mark.parametrize("cs", [2, 4, 8, 16])
def test_twolevel_pass_matches_oracle_for_every_cluster_size(case, cs, precision, mode):
    op, buf, Theta, grad = run_pass(case, mode, cs, precision)
    assert op.plan(1, 1)["cs"] == cs
    check(case, op, buf, Theta, grad)


@pytest.mark.parametrize("mode", MODES)
def test_twolevel_fp64_path_keeps_the_fp64_tolerance(case, mode):
    """FP64 CG with the two-level coarse correction (applied in FP32, refined in FP64)."""
    op, buf, Theta, grad = run_pass(case, mode, 0, "fp64")
    check(case, op, buf, Theta, grad, FP64_TOL, FP64_TOL)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("precision", ["fp32_refine", "fp32_refine_all"])
def test_twolevel_reduces_coarse_iterations(case, precision, mode):
    on = run_pass(case, mode, 0, precision)
    off = run_pass(case, "none", 0, precision)
    check(case, *on)
    check(case, *off)
    k_on, k_off = on[0].stats()["by_kind"], off[0].stats()["by_kind"]
    for name in ("coarse_primal", "correct_primal", "coarse_adjoint", "correct_adjoint"):
        assert k_on[name]["solves"] == k_off[name]["solves"] > 0
        assert k_on[name]["cg_iters"] < 0.8 * k_off[name]["cg_iters"], (name, k_on[name], k_off[name])
    for name in ("fine_primal", "fine_adjoint"):      # fine solves keep Jacobi (the adjoint
        assert k_on[name]["solves"] == k_off[name]["solves"]  # source moves with Theta's rounding)
        assert abs(k_on[name]["cg_iters"] - k_off[name]["cg_iters"]) <= 0.01 * k_off[name]["cg_iters"]


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine", "fp32_refine_all"])
def test_vcycle_needs_fewer_iterations_than_additive(case, precision):
    """Coarse-step solves: the two-grid cycle's smoothing removes the high-frequency error
    that the additive form leaves to CG (an iteration-count check, as above)."""
    runs = {m: run_pass(case, m, 0, precision) for m in MODES}
    tol = FP64_TOL if precision == "fp64" else None
    for m in MODES:
        if tol:
            check(case, *runs[m], tol, tol)
        else:
            check(case, *runs[m])
    k = {m: runs[m][0].stats()["by_kind"] for m in MODES}
    for name in ("coarse_primal", "correct_primal", "coarse_adjoint", "correct_adjoint"):
        assert k["vcycle1"][name]["cg_iters"] < 0.75 * k["additive"][name]["cg_iters"], (name, k)
        assert k["vcycle3"][name]["cg_iters"] < 0.9 * k["vcycle1"][name]["cg_iters"], (name, k)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine_all"])
@pytest.mark.parametrize("design", ["branches_table1_bottom", "uniform_simp_left"])
def test_twolevel_helps_on_high_contrast_designs(design, precision, mode):
    """The preconditioner must pay on a near-binary design too (an iteration-count check: the
    parity tests pass even with a useless preconditioner, because CG still converges)."""
    from paper_2411_19030_gb300 import parareal_pass
    n, Nt = 64, 256
    if design == "branches_table1_bottom":
        prob, rho = make_problem(n, Nt=Nt, Ntau=16, dt=1 / Nt, material="table1", sink="bottom"), W.rho_branches(n, n)
    else:
        prob, rho = make_problem(n, Nt=Nt, Ntau=16, dt=1 / Nt), W.rho_uniform(n, n, 1, 0.2, 0.8)
    its = {}
    smooth = int(mode[6:]) if mode.startswith("vcycle") else 0
    for tl in (mode, "none"):
        op = gpu_operator(prob, precision, rtol=1e-10, twolevel=tl[:6] if tl.startswith("vcycle") else tl,
                          smooth_steps=smooth if tl == mode else 0)
        buf = PassBuffers(op)
        op.assemble(dev(rho))
        parareal_pass(op, buf, 1)
        torch.cuda.synchronize()
        assert op.stats()["status"] == 0
        # the correction sweeps: the initial coarse sweep (from zero) and the iteration's
        # sweep.  The batched G of the iteration starts from u_{s+1}^0 = G(u_s^0) itself
        # (ptg_solve.initial_guess) and takes no iteration at all here.
        st = op.stats()["by_kind"]["correct_primal"]
        its[tl] = st["cg_iters"] / st["solves"]
    assert its[mode] < 0.6 * its["none"], its


@pytest.mark.parametrize("precision", ["fp32_refine", "fp32_refine_all"])
def test_slab_local_two_step_preconditioner_of_the_fine_solves(case, precision):
    """local_steps = 2: the FP32 fine-step CG preconditioned by two damped-Jacobi steps on each
    CTA's slab; the pass still matches the oracle, with fewer fine CG iterations than Jacobi."""
    prob, rho, U_old, V_old, _ = case
    out = {}
    for steps in (1, 2):
        op = gpu_operator(prob, precision, rtol=1e-10, local_steps=steps)
        buf = PassBuffers(op)
        buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
        buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
        op.assemble(dev(rho))
        Theta, grad = oneshot_pass(op, buf)
        torch.cuda.synchronize()
        check(case, op, buf, Theta, grad)
        out[steps] = op.stats()["by_kind"]
    for name in ("fine_primal", "fine_adjoint"):
        assert out[2][name]["cg_iters"] < 0.9 * out[1][name]["cg_iters"], (name, out)
