"""Failure detection on the device without faulting it: the bounded wait of a grid barrier is
made to run out (ptg_op_set_wait_limit with a limit of one poll), so the cooperative launch
records PTG_ETIMEOUT in the op's status word and every CTA stops waiting and returns.  The
error is read on the host through ptg_get_stats; after ptg_reset_stats and the default limit
the same op gives the oracle's result again.  Nothing here traps or hangs the GPU: every wait is
bounded and every loop of the stepper has an iteration limit."""
from __future__ import annotations

import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp, sequential_pass as o_sequential
from paper_2411_19030_gb300 import PassBuffers, sequential_pass
from paper_2411_19030_gb300._ffi import PTG_ETIMEOUT
from tests.gpu_helpers import FP64_TOL, assert_close, dev, ensure_built, gpu_operator, host
from tests.problems import make_problem

pytestmark = pytest.mark.gpu


def test_grid_barrier_wait_limit_reports_timeout_and_op_recovers():
    ensure_built()
    prob = make_problem(13, 9, Nt=24, Ntau=4, dt=1 / 24, material="table1", sink="left_wide",
                        q_time=W.q_time_paper(24, 1 / 24))
    rho = W.rho_uniform(13, 9, 3, 0.05, 0.95)
    seq = o_sequential(OracleOp(prob, rho))
    # small iteration limits: once the barrier is broken the reductions are meaningless and the
    # solves run to their limits, which keeps the broken launch short
    op = gpu_operator(prob, "fp64", grid_wide=2, cg_iters_max=40, refine_max=2)
    assert op.plan(0, 1)["cs"] > 1          # a cooperative grid of several CTAs per system
    buf = PassBuffers(op)
    op.assemble(dev(rho))
    op.set_wait_limit(1)
    sequential_pass(op, buf)
    torch.cuda.synchronize()
    st = op.stats()
    assert st["status"] == PTG_ETIMEOUT, st
    assert st["fail_kind"] in (10, 13), st   # recorded by a fine primal or fine adjoint launch
    # the context is intact and the op recovers with the default limit
    op.set_wait_limit(0)
    op.reset_stats()
    op2 = gpu_operator(prob, "fp64", grid_wide=2)
    for o in (op, op2):
        o.set_wait_limit(0)
    op.close()
    b2 = PassBuffers(op2)
    op2.assemble(dev(rho))
    Theta, grad = sequential_pass(op2, b2)
    torch.cuda.synchronize()
    assert_close("T_hist after recovery", host(b2.T_hist), seq["T_hist"], FP64_TOL)
    assert_close("grad after recovery", host(grad), seq["grad"], FP64_TOL)
    assert op2.stats()["status"] == 0


def test_wait_limit_rejects_negative_values():
    ensure_built()
    prob = make_problem(6, Nt=4, Ntau=2, dt=0.25)
    op = gpu_operator(prob, "fp64")
    with pytest.raises(Exception):
        op.set_wait_limit(-1)
