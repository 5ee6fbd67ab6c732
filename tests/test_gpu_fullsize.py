"""Parity at the full sizes of the measured configurations, in the launch configuration that
bench.py times (the default plans of the library), on outputs the oracle can produce in
seconds or through properties that hold at any size.

* 128 x 128, Nt = 1024, N_tau = 32 (the benchmark workload): the whole one-shot pass against
  the oracle's one-shot pass (about 20 s of CPU).
* 256 x 256, Nt = 2048, N_tau = 64, rho ~ U(0, 1) seed 1 (differentiation): the checkpointed
  autograd gradient against the full-history GPU gradient; central differences of the FP64
  GPU forward along a random direction over the 32 elements of the configuration and on 4
  single elements; the backward's extra device memory against the full history's size.
* 48 designs of uneven size (batching): one batched one-shot pass against single-design
  passes, the CUDA-graph replay bit for bit, and the smallest design against the oracle.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp
from oracle import coarse_states_from_sequential, oneshot_pass as o_oneshot
from paper_2411_19030_gb300 import PassBuffers, oneshot_pass, sequential_pass
from paper_2411_19030_gb300.autograd import ParaTopoFn, forward_checkpointed
from paper_2411_19030_gb300.batch import Batch
from tests.gpu_helpers import (FP64_TOL, MIXED_G_TOL, MIXED_T_TOL, assert_close, dev, ensure_built, gpu_operator,
                               host, rel_err)
from tests.problems import make_problem

pytestmark = pytest.mark.gpu

BENCH_SOLVE = dict(rtol=1e-10, inner_rtol=1e-4, cg_iters_max=2000, refine_max=8)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def workload(name):
    w = W.workload(name)
    return make_problem(w["n"], Nt=w["Nt"], Ntau=w["Ntau"], dt=w["dt"], p=w["p"]), w


def test_oneshot128_pass_matches_oracle():
    prob, _ = workload("oneshot128")
    rho_old = W.rho_uniform(128, 128, 0, 0.2, 0.8)
    rho = W.rho_warm_perturb(rho_old, seed=1000, amp=0.01)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    op = gpu_operator(prob, "fp32_refine", **BENCH_SOLVE)
    buf = PassBuffers(op)
    buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
    buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
    op.assemble(dev(rho))
    Theta, grad = oneshot_pass(op, buf)
    torch.cuda.synchronize()
    assert_close("T_hist", host(buf.T_hist), ref["T_hist"], MIXED_T_TOL)
    assert_close("U_new", host(buf.U_T_new), ref["U"][0], MIXED_T_TOL)
    assert_close("Theta", host(Theta), [ref["Theta"]], MIXED_T_TOL)
    assert_close("V_lam", host(buf.V_l_new), ref["V"][0], MIXED_G_TOL)
    assert_close("grad", host(grad), ref["grad"], MIXED_G_TOL)
    assert op.stats()["status"] == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_loop512_grouped_pass_matches_oracle_on_a_short_time_grid(precision):
    """512 x 512 with the design loop's step size (dt = 1/4096), on a short time grid (Nt = 64 in
    8 slices): no slab of this grid fits a 16-CTA cluster, so every kind runs in groups of a
    cooperative launch, as in the full 512 x 512 loop.  The one-shot pass against the oracle's,
    element by element (warm start of a design 1% away)."""
    prob = make_problem(512, Nt=64, Ntau=8, dt=1 / 4096)
    rho = W.rho_uniform(512, 512, 5, 0.2, 0.8)
    rho_old = W.rho_warm_perturb(rho, seed=6, amp=0.01)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
    fp64 = precision == "fp64"
    # FP64: rtol 1e-12, the floor of the FP64 coarse-step CG with an FP32 preconditioner
    op = gpu_operator(prob, precision, **dict(BENCH_SOLVE, rtol=1e-12 if fp64 else 1e-10))
    assert op.plan(0, 8)["cs"] > 16 and op.plan(2, 1)["cs"] > 16
    buf = PassBuffers(op)
    buf.U_T.copy_(dev(U_old[0])); buf.U_th.copy_(dev(U_old[1]))
    buf.V_l.copy_(dev(V_old[0])); buf.V_g.copy_(dev(V_old[1]))
    op.assemble(dev(rho))
    Theta, grad = oneshot_pass(op, buf)
    torch.cuda.synchronize()
    tol_t, tol_g = (FP64_TOL, FP64_TOL) if fp64 else (MIXED_T_TOL, MIXED_G_TOL)
    assert_close("T_hist", host(buf.T_hist), ref["T_hist"], tol_t)
    assert_close("U_new", host(buf.U_T_new), ref["U"][0], tol_t)
    assert_close("Theta", host(Theta), [ref["Theta"]], tol_t)
    assert_close("V_lam", host(buf.V_l_new), ref["V"][0], tol_g)
    assert_close("grad", host(grad), ref["grad"], tol_g)
    assert op.stats()["status"] == 0, op.stats()


def test_diff256_autograd_gradient():
    prob, _ = workload("diff256")
    rho_np = W.rho_uniform(256, 256, 1, 0.0, 1.0)
    op = gpu_operator(prob, "fp64", rtol=1e-13)
    # checkpointed autograd gradient, with its extra device memory
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    rho = dev(rho_np).requires_grad_(True)
    ParaTopoFn.apply(rho, op).sum().backward()
    torch.cuda.synchronize()
    extra = torch.cuda.max_memory_allocated() - base
    g = host(rho.grad).copy()
    history = (prob.Nt + 1) * prob.Nn * 8
    assert extra < 0.25 * history, (extra, history)
    # the same gradient from the full-history sequential pass
    buf = PassBuffers(op)
    op.assemble(dev(rho_np))
    Theta, grad = sequential_pass(op, buf)
    torch.cuda.synchronize()
    assert_close("checkpointed vs full history", g, host(grad), 1e-12)
    assert op.stats()["status"] == 0
    # central differences of the FP64 forward on the configuration's 32 elements
    elems = W.fd_elements(prob.Ne, 32, seed=1)
    # step 1e-5: the difference quotient's error from the solves is about rtol * Theta / eps
    # (each forward meets rtol 1e-13 on its own, from its own CG starts), the truncation error
    # O(eps^2) stays far below the bound
    eps = 1e-5
    assert np.all((rho_np[elems] > eps) & (rho_np[elems] < 1 - eps))
    gmax = float(np.max(np.abs(g)))

    def theta(r):
        return float(forward_checkpointed(op, dev(r))[0].item())

    d = np.random.default_rng(5).choice([-1.0, 1.0], size=32)
    rp, rm = rho_np.copy(), rho_np.copy()
    rp[elems] += eps * d
    rm[elems] -= eps * d
    fd_dir = (theta(rp) - theta(rm)) / (2 * eps)
    assert abs(fd_dir - float(np.dot(g[elems], d))) <= 1e-6 * gmax * np.sqrt(32), (fd_dir, np.dot(g[elems], d))
    for e in elems[:4]:
        rp, rm = rho_np.copy(), rho_np.copy()
        rp[e] += eps
        rm[e] -= eps
        fd = (theta(rp) - theta(rm)) / (2 * eps)
        assert abs(fd - g[e]) <= 1e-6 * gmax, (e, fd, g[e], gmax)


def test_batch48_pass():
    designs = W.batch48()
    probs = [make_problem(d["n"], Nt=d["Nt"], Ntau=d["Ntau"], dt=d["dt"], p=d["p"]) for d in designs]
    ops = [gpu_operator(p, "fp32_refine", **BENCH_SOLVE) for p in probs]
    batch = Batch(ops)
    rho_old = [W.rho_warm_perturb(d["rho"], seed=1000 + d["index"], amp=0.01) for d in designs]
    # warm start: the sequential pass of the previous designs, then the one-shot pass
    for i in range(48):
        batch.buffers(i)["rho"].copy_(dev(rho_old[i]))
    batch.assemble()
    batch.sequential_pass()
    for i, d in enumerate(designs):
        batch.buffers(i)["rho"].copy_(dev(d["rho"]))
    batch.assemble()
    batch.oneshot_pass()
    torch.cuda.synchronize()
    res = [(host(batch.buffers(i)["T_hist"][::97]).copy(), host(batch.buffers(i)["U_theta_new"]).copy(),
            host(batch.buffers(i)["V_g_new"][0]).copy()) for i in range(48)]
    for op in ops:
        assert op.stats()["status"] == 0
    # CUDA graph of assembly + pass, replayed: bit for bit the direct pass
    for i in range(48):
        batch.buffers(i)["V_g_new"].zero_()
    batch.capture()
    batch.replay()
    torch.cuda.synchronize()
    for i in range(48):
        assert np.array_equal(host(batch.buffers(i)["V_g_new"][0]), res[i][2]), i
    # one design of each size against single-design passes of the same library (other plans)
    for i in range(5):
        op1 = gpu_operator(probs[i], "fp32_refine", **BENCH_SOLVE)
        b1 = PassBuffers(op1)
        op1.assemble(dev(rho_old[i]))
        sequential_pass(op1, b1)
        op1.assemble(dev(designs[i]["rho"]))
        Th, gr = oneshot_pass(op1, b1)
        torch.cuda.synchronize()
        assert rel_err(host(b1.T_hist[::97]), res[i][0]) < 1e-8, i
        assert rel_err(host(b1.U_th_new), res[i][1]) < 1e-8, i
        assert rel_err(host(gr), res[i][2]) < 1e-7, i
        del b1, op1
    # the smallest design (64 x 64, Nt = 512) against the oracle
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(probs[0], rho_old[0]))
    ref = o_oneshot(OracleOp(probs[0], designs[0]["rho"]), U_old, V_old)
    assert_close("Theta[0]", res[0][1][probs[0].Ntau:], [ref["Theta"]], MIXED_T_TOL)
    assert_close("grad[0]", res[0][2], ref["grad"], MIXED_G_TOL)
    batch.close()
