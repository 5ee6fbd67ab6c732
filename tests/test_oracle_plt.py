"""Pins of the oracle's modified objective Theta~ = Theta^p and of the PLT variant
(coarse propagators identically zero), Sec. 7.  CPU only."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from oracle import Operator, coarse_states_from_sequential, objective_from_modified, oneshot_pass, parareal, sequential_pass
from tests.problems import make_problem


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def pair(modified, **kw):
    base = dict(Nt=12, Ntau=4, dt=0.04, material="table1", sink="left_wide", q_time=W.q_time_paper(12, 0.04))
    base.update(kw)
    return make_problem(6, 5, modified_objective=modified, **base)


RHO = W.rho_uniform(6, 5, 21, 0.1, 0.9)


@pytest.mark.parametrize("p", [8.0, 20.0])
def test_modified_objective_is_theta_to_the_p(p):
    """Sec. 7.1: Theta~ = Theta^p, and the cumulative objectives obey theta~_j = theta_j^p."""
    a = sequential_pass(Operator(pair(False, p=p), RHO))
    b = sequential_pass(Operator(pair(True, p=p), RHO))
    assert abs(b["Theta"] - a["Theta"] ** p) <= 1e-13 * b["Theta"]
    assert rel(b["theta"][1:], a["theta"][1:] ** p) < 1e-13
    assert rel(b["T_hist"], a["T_hist"]) == 0.0          # the state does not depend on the objective


@pytest.mark.parametrize("p", [8.0, 20.0])
def test_gradient_identity_between_the_objectives(p):
    """Sec. 7.1: grad Theta = Theta^(1-p)/p grad Theta~, with the adjoint source p/Ne T^(p-1)
    for Theta~ against Theta^(1-p)/Ne T^(p-1) for Theta."""
    a = sequential_pass(Operator(pair(False, p=p), RHO))
    b = sequential_pass(Operator(pair(True, p=p), RHO))
    Theta, grad = objective_from_modified(b["Theta"], b["grad"], p)
    assert abs(Theta - a["Theta"]) <= 1e-14 * a["Theta"]
    assert rel(grad, a["grad"]) < 1e-12
    # the two gradients differ by the factor p Theta^(p-1), far from 1: the check is not vacuous
    assert rel(b["grad"], a["grad"]) > 0.5


def test_modified_gradient_matches_central_differences():
    """The adjoint of Theta~ against central differences (eps = 1e-6) on every element,
    capacity SIMP active (the dC/drho term of Eq. 4.7)."""
    prob = make_problem(5, 4, Nt=8, dt=0.06, material="table1", sink="left_wide", p=8.0,
                        q_time=W.q_time_paper(8, 0.06), modified_objective=True)
    rho = W.rho_uniform(5, 4, 7, 0.15, 0.85)
    g = sequential_pass(Operator(prob, rho))["grad"]
    eps = 1e-6
    fd = np.zeros_like(g)
    for e in range(prob.Ne):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += eps
        rm[e] -= eps
        fd[e] = (sequential_pass(Operator(prob, rp))["Theta"] - sequential_pass(Operator(prob, rm))["Theta"]) / (2 * eps)
    assert rel(g, fd) < 1e-6


@pytest.mark.parametrize("modified", [False, True])
def test_plt_fixed_point_and_correction_is_F(modified):
    """Eq. 7.2: with G = 0 the corrected states are the fine results of the old states, so a
    warm start from the exact sequential coarse states reproduces the sequential pass."""
    prob = pair(modified)
    op = Operator(prob, RHO)
    U, V, seq = coarse_states_from_sequential(op)
    out = oneshot_pass(op, U, V, plt=True)
    assert np.array_equal(out["U"][0][1:], out["F_pri"][0])
    assert np.array_equal(out["U"][1][1:], out["F_pri"][1])
    assert np.array_equal(out["V"][0][:-1], out["F_adj"][0])
    assert np.array_equal(out["V"][1][:-1], out["F_adj"][1])
    assert np.all(out["G_pri_old"][0] == 0) and np.all(out["G_adj_old"][1] == 0)
    assert rel(out["T_hist"], seq["T_hist"]) < 1e-13
    assert abs(out["Theta"] - seq["Theta"]) <= 1e-13 * seq["Theta"]
    assert rel(out["grad"], seq["grad"]) < 1e-12


@pytest.mark.parametrize("Nt,Ntau", [(12, 4), (12, 3), (6, 1)])
def test_plt_exact_after_Ntau_iterations(Nt, Ntau):
    """With G = 0, iteration k fixes slices 0..k-1 exactly (each starts from an exact state), so
    N_tau iterations reproduce the sequential run; one iteration does not (unless N_tau = 1)."""
    prob = pair(True, Nt=Nt, Ntau=Ntau, dt=0.5 / Nt, q_time=W.q_time_paper(Nt, 0.5 / Nt))
    op = Operator(prob, RHO)
    seq = sequential_pass(op)
    par = parareal(op, Ntau, plt=True)
    assert rel(par["T_hist"], seq["T_hist"]) < 1e-12
    assert abs(par["Theta"] - seq["Theta"]) <= 1e-12 * seq["Theta"]
    assert rel(par["grad"], seq["grad"]) < 1e-11
    if Ntau > 1:
        assert rel(parareal(op, 1, plt=True)["grad"], seq["grad"]) > 1e-6
