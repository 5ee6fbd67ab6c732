"""Differentiation (ParaTopoFn): the gradient from the checkpointed adjoint matches the oracle's
discrete-adjoint gradient and central finite differences of the GPU forward, and the backward
recomputes each slice from its checkpoint with bounded memory."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle import Operator as OracleOp, sequential_pass as o_sequential
from paper_2411_19030_gb300.autograd import ParaTopoFn, backward_checkpointed, forward_checkpointed
from tests.gpu_helpers import FP64_TOL, assert_close, dev, ensure_built, gpu_operator, host
from tests.problems import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("material,Ntau", [("table1", 4), ("simp_k", 8), ("simp_k", 1)])
def test_autograd_gradient_matches_oracle(material, Ntau):
    Nt = 24
    prob = make_problem(15, 10, Nt=Nt, Ntau=Ntau, dt=1 / Nt, material=material, sink="left_wide",
                        q_time=W.q_time_paper(Nt, 1 / Nt))
    rho_np = W.rho_uniform(15, 10, 21, 0.05, 0.95)
    seq = o_sequential(OracleOp(prob, rho_np))
    op = gpu_operator(prob)
    rho = dev(rho_np).requires_grad_(True)
    Theta = ParaTopoFn.apply(rho, op)
    assert_close("Theta", host(Theta.detach()), [seq["Theta"]], FP64_TOL)
    (3.0 * Theta).sum().backward()
    assert_close("grad", host(rho.grad), 3.0 * seq["grad"], FP64_TOL)
    assert op.stats()["status"] == 0


def test_autograd_matches_central_differences_of_the_gpu_forward():
    """Central differences (eps = 1e-5) of the GPU forward on 12 elements, FP64."""
    Nt = 40
    prob = make_problem(16, Nt=Nt, Ntau=5, dt=0.5 / Nt, material="table1", sink="left_wide", p=8.0)
    rho_np = W.rho_uniform(16, 16, 4, 0.1, 0.9)
    op = gpu_operator(prob)
    rho = dev(rho_np).requires_grad_(True)
    ParaTopoFn.apply(rho, op).sum().backward()
    g = host(rho.grad)
    eps = 1e-5
    gmax = np.max(np.abs(g))
    for e in W.fd_elements(prob.Ne, 12, seed=9):
        rp, rm = rho_np.copy(), rho_np.copy()
        rp[e] += eps
        rm[e] -= eps
        tp = float(forward_checkpointed(op, dev(rp))[0].item())
        tm = float(forward_checkpointed(op, dev(rm))[0].item())
        fd = (tp - tm) / (2 * eps)
        assert abs(fd - g[e]) <= 1e-6 * gmax, (e, fd, g[e], gmax)


def test_checkpointed_backward_memory_is_bounded():
    """The backward holds (Ntau+1) + (M+1) node vectors, not the (Nt+1)-row history."""
    Nt, Ntau = 64, 8
    prob = make_problem(12, Nt=Nt, Ntau=Ntau, dt=1 / Nt)
    op = gpu_operator(prob)
    rho = dev(W.rho_uniform(12, 12, 2, 0.2, 0.8))
    _, ck = forward_checkpointed(op, rho)
    rows = ck.U_T.shape[0] + ck.window.shape[0]
    assert rows == (Ntau + 1) + (Nt // Ntau + 1) and rows < Nt + 1
    g = backward_checkpointed(op, ck)
    seq = o_sequential(OracleOp(prob, host(rho)))
    assert_close("grad", host(g), seq["grad"], FP64_TOL)
