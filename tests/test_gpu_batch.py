"""Batching: designs of different grid sizes, time grids and slice counts advanced together
(one persistent launch per phase), against the oracle design by design; the CUDA-graph replay
of a whole batched pass; the autotuner."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp
from oracle import coarse_states_from_sequential, oneshot_pass as o_oneshot, sequential_pass as o_sequential
from paper_2411_19030_gb300.batch import Batch, autotune
from tests.gpu_helpers import FP64_TOL, MIXED_G_TOL, MIXED_T_TOL, assert_close, dev, ensure_built, gpu_operator, host
from tests.problems import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def designs():
    """Uneven sizes (the batching workload scaled down): grids 16..40, Nt 24..60, N_tau 3..6."""
    out = []
    specs = [(24, 24, 48, 6, "simp_k", "left"), (16, 16, 24, 4, "table1", "left_wide"),
             (40, 40, 60, 5, "simp_k", "left"), (13, 9, 24, 3, "table1", "left_wide"),
             (32, 32, 40, 4, "simp_k", "left")]
    for i, (nx, ny, Nt, Ntau, mat, sink) in enumerate(specs):
        prob = make_problem(nx, ny, Nt=Nt, Ntau=Ntau, dt=1.0 / Nt, material=mat, sink=sink,
                            q_time=W.q_time_paper(Nt, 1.0 / Nt) if mat == "table1" else None)
        out.append((prob, W.rho_uniform(nx, ny, 100 + i, 0.05, 0.95)))
    return out


def make_batch(precision="fp64", **kw):
    ds = designs()
    ops = [gpu_operator(p, precision, **kw) for p, _ in ds]
    return ds, ops, Batch(ops)


def test_batched_sequential_pass_matches_oracle_per_design():
    ds, ops, batch = make_batch()
    for d, (_, rho) in enumerate(ds):
        batch.buffers(d)["rho"].copy_(dev(rho))
    batch.assemble()
    batch.sequential_pass()
    torch.cuda.synchronize()
    for d, (prob, rho) in enumerate(ds):
        seq = o_sequential(OracleOp(prob, rho))
        b = batch.buffers(d)
        assert_close(f"T_hist[{d}]", host(b["T_hist"]), seq["T_hist"], FP64_TOL)
        assert_close(f"Theta[{d}]", host(b["U_theta"][prob.Ntau:]), [seq["Theta"]], FP64_TOL)
        assert_close(f"grad[{d}]", host(b["V_g"][0]), seq["grad"], FP64_TOL)
    for op in ops:
        assert op.stats()["status"] == 0


@pytest.mark.parametrize("precision,tol_t,tol_g", [("fp64", FP64_TOL, FP64_TOL),
                                                   ("fp32_refine", MIXED_T_TOL, MIXED_G_TOL),
                                                   ("fp32_refine_all", MIXED_T_TOL, MIXED_G_TOL)])
def test_batched_oneshot_pass_matches_oracle_per_design(precision, tol_t, tol_g):
    kw = {} if precision == "fp64" else {"rtol": 1e-10}
    ds, ops, batch = make_batch(precision, **kw)
    refs = []
    for d, (prob, rho) in enumerate(ds):
        rho_old = W.rho_warm_perturb(rho, seed=200 + d, amp=0.05)
        U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
        refs.append(o_oneshot(OracleOp(prob, rho), U_old, V_old))
        b = batch.buffers(d)
        b["U_T"].copy_(dev(U_old[0])); b["U_theta"].copy_(dev(U_old[1]))
        b["V_lam"].copy_(dev(V_old[0])); b["V_g"].copy_(dev(V_old[1]))
        b["rho"].copy_(dev(rho))
    batch.assemble()
    batch.oneshot_pass()
    torch.cuda.synchronize()
    for d, (prob, _) in enumerate(ds):
        b, ref = batch.buffers(d), refs[d]
        assert_close(f"T_hist[{d}]", host(b["T_hist"]), ref["T_hist"], tol_t)
        assert_close(f"U_new[{d}]", host(b["U_T_new"]), ref["U"][0], tol_t)
        assert_close(f"Theta[{d}]", host(b["U_theta_new"][prob.Ntau:]), [ref["Theta"]], tol_t)
        assert_close(f"V_new[{d}]", host(b["V_lam_new"]), ref["V"][0], tol_g)
        assert_close(f"grad[{d}]", host(b["V_g_new"][0]), ref["grad"], tol_g)


def test_graph_replay_reproduces_the_batched_pass_bit_for_bit():
    ds, ops, batch = make_batch("fp32_refine", rtol=1e-10)
    for d, (_, rho) in enumerate(ds):
        batch.buffers(d)["rho"].copy_(dev(rho))
    batch.assemble()
    batch.sequential_pass()       # warm start = sequential states of the same designs
    batch.assemble()
    batch.oneshot_pass()
    torch.cuda.synchronize()
    direct = [host(batch.buffers(d)["V_g_new"][0]).copy() for d in range(len(ds))]
    batch.capture()
    for d in range(len(ds)):
        batch.buffers(d)["V_g_new"].zero_()
    batch.replay()
    torch.cuda.synchronize()
    for d in range(len(ds)):
        assert np.array_equal(host(batch.buffers(d)["V_g_new"][0]), direct[d])


def test_autotuner_installs_valid_plans_and_keeps_results():
    ds, ops, batch = make_batch()
    for d, (_, rho) in enumerate(ds):
        batch.buffers(d)["rho"].copy_(dev(rho))
    batch.assemble()
    batch.sequential_pass()
    res = autotune(batch, phases=range(6), reps=1)
    assert set(res) == {"fine_primal", "coarse_primal", "correct_primal", "fine_adjoint", "coarse_adjoint",
                        "correct_adjoint"}
    for ph in range(6):
        p = batch.plan(ph)
        assert p["cs"] in (2, 4, 8, 16) and 1 <= p["ng"] <= 6 and p["nclusters"] >= 1
    batch.oneshot_pass()          # warm start = exact sequential states: the fixed point
    torch.cuda.synchronize()
    for d, (prob, rho) in enumerate(ds):
        seq = o_sequential(OracleOp(prob, rho))
        assert_close(f"grad[{d}]", host(batch.buffers(d)["V_g_new"][0]), seq["grad"], FP64_TOL)


# ---------------------------------------------------------------- designs on their own path

def make_mixed_batch(precision="fp64", **kw):
    """The same designs, the even ones (24^2, 40^2, 32^2) with streamed coarse-step solves
    (coarse_stream = 2): the batch runs those through their ops' own launches and the rest in the
    persistent launches."""
    ds = designs()
    ops = [gpu_operator(p, precision, coarse_stream=2 if d in (0, 2, 4) else 1, **kw) for d, (p, _) in enumerate(ds)]
    return ds, ops, Batch(ops)


def _warm(ds, batch, seed):
    refs = []
    for d, (prob, rho) in enumerate(ds):
        rho_old = W.rho_warm_perturb(rho, seed=seed + d, amp=0.05)
        U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
        refs.append((U_old, V_old))
        b = batch.buffers(d)
        b["U_T"].copy_(dev(U_old[0])); b["U_theta"].copy_(dev(U_old[1]))
        b["V_lam"].copy_(dev(V_old[0])); b["V_g"].copy_(dev(V_old[1]))
        b["rho"].copy_(dev(rho))
    return refs


@pytest.mark.parametrize("precision,tol_t,tol_g", [("fp64", FP64_TOL, FP64_TOL),
                                                   ("fp32_refine", MIXED_T_TOL, MIXED_G_TOL)])
@pytest.mark.parametrize("plt", [False, True])
def test_batch_with_designs_on_their_own_path_matches_oracle(precision, tol_t, tol_g, plt):
    from paper_2411_19030_gb300 import PassBuffers, oneshot_pass
    kw = {"rtol": 1e-12} if precision == "fp64" else {"rtol": 1e-10}
    ds, ops, batch = make_mixed_batch(precision, **kw)
    warm = _warm(ds, batch, 300)
    batch.assemble()
    batch.oneshot_pass(plt=plt)
    torch.cuda.synchronize()
    for d, (prob, rho) in enumerate(ds):
        U_old, V_old = warm[d]
        ref = o_oneshot(OracleOp(prob, rho), U_old, V_old, plt=plt)
        b = batch.buffers(d)
        assert_close(f"T_hist[{d}]", host(b["T_hist"]), ref["T_hist"], tol_t)
        assert_close(f"U_new[{d}]", host(b["U_T_new"]), ref["U"][0], tol_t)
        assert_close(f"Theta[{d}]", host(b["U_theta_new"][prob.Ntau:]), [ref["Theta"]], tol_t)
        assert_close(f"V_new[{d}]", host(b["V_lam_new"]), ref["V"][0], tol_g)
        assert_close(f"grad[{d}]", host(b["V_g_new"][0]), ref["grad"], tol_g)
    for op in ops:
        assert op.stats()["status"] == 0
    # a design on its own path equals the single-design pass of its op, bit for bit, with the
    # sweep group the batch gives it (16 CTAs: the batch runs its large designs' sweeps side by side)
    d = 2
    op, b = ops[d], batch.buffers(d)
    G = min(16, (op.ny + 1) // 2)
    op.set_plan(2, G)
    op.set_plan(5, G)
    buf = PassBuffers(op)
    U_old, V_old = warm[d]
    buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
    buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
    op.assemble(b["rho"].clone())
    oneshot_pass(op, buf, plt=plt, overlap=False)
    torch.cuda.synchronize()
    assert torch.equal(buf.T_hist, b["T_hist"]) and torch.equal(buf.V_g_new, b["V_g_new"])
    op.set_plan(2, 0)
    op.set_plan(5, 0)


def test_graph_replay_of_a_batch_with_designs_on_their_own_path():
    ds, ops, batch = make_mixed_batch("fp32_refine", rtol=1e-10)
    assert [batch.own_path(d) for d in range(len(ds))] == [True, False, True, False, True]
    for d, (_, rho) in enumerate(ds):
        batch.buffers(d)["rho"].copy_(dev(rho))
    batch.assemble()
    batch.sequential_pass()
    batch.assemble()
    batch.oneshot_pass()
    torch.cuda.synchronize()
    direct = [host(batch.buffers(d)["V_g_new"][0]).copy() for d in range(len(ds))]
    batch.capture()
    for d in range(len(ds)):
        batch.buffers(d)["V_g_new"].zero_()
    batch.replay()
    torch.cuda.synchronize()
    for d in range(len(ds)):
        assert np.array_equal(host(batch.buffers(d)["V_g_new"][0]), direct[d])
