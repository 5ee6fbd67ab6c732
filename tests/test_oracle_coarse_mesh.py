"""Pins of the oracle's coarse-mesh propagators (the future work of Sec. 7.3): the transfers
against closed forms, the coarse operators against the Galerkin products that nested
bilinear spaces imply, Galerkin orthogonality of a coarse step, Parareal's exactness and the
one-shot fixed point with the coarse-mesh G, and the second-order consistency of the coarse
step with the fine one.  CPU only."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from oracle import Operator, coarse_states_from_sequential, oneshot_pass, parareal, sequential_pass
from oracle.coarse_mesh import CoarseMesh, coarse_elements, injection, prolongation
from oracle.fem import assemble
from oracle.parareal import G_pri
from tests.problems import make_problem


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def nodes(n, m, h):
    y, x = np.divmod(np.arange((n + 1) * (m + 1)), m + 1)
    return x * h, y * h


def test_prolongation_reproduces_bilinear_fields_and_injection_inverts_it():
    prob = make_problem(8, 6, Nt=4, Ntau=2, sink="none")
    xH, yH = nodes(3, 4, 2 * prob.h)
    xh, yh = nodes(6, 8, prob.h)
    f = lambda x, y: 0.3 + 1.7 * x - 0.9 * y + 2.3 * x * y
    P = prolongation(prob)
    assert rel(P @ f(xH, yH), f(xh, yh)) < 1e-15
    c = W.rho_uniform(5, 4, 3, -1.0, 1.0)
    assert rel(injection(prob, P @ c), c) == 0.0


def test_restricted_fine_load_is_the_coarse_load():
    """For nested bilinear spaces and a uniform source, P^T f_h is the load assembled on 2h."""
    prob = make_problem(8, 6, Nt=4, Ntau=2, sink="none")
    cm = CoarseMesh(Operator(prob, np.full(prob.Ne, 0.5)))
    assert rel(cm.P.T @ Operator(prob, np.full(prob.Ne, 0.5)).f, cm.opH.f) < 1e-14


@pytest.mark.parametrize("material", ["simp_k", "table1"])
def test_coarse_operators_are_the_galerkin_products_for_a_uniform_design(material):
    prob = make_problem(8, 6, Nt=4, Ntau=2, sink="none", material=material)
    rho = np.full(prob.Ne, 0.37)
    cm = CoarseMesh(Operator(prob, rho))
    K, C, _ = assemble(prob, rho)
    P = cm.P
    assert rel((P.T @ K @ P).toarray(), cm.opH.K.toarray()) < 1e-13
    assert rel((P.T @ C @ P).toarray(), cm.opH.C.toarray()) < 1e-13


def test_coarse_design_is_the_mean_of_the_children():
    v = np.arange(24, dtype=np.float64)          # 6 x 4 elements
    out = coarse_elements(v, 6, 4)
    assert np.array_equal(out, [3.5, 5.5, 7.5, 15.5, 17.5, 19.5])


def test_coarse_primal_step_is_galerkin_orthogonal_on_nested_states():
    """For a uniform design and a state in range(P), G_pri returns P x with
    P^T (A P x - b) = 0: the energy-norm best approximation of the fine coarse step."""
    prob = make_problem(10, 8, Nt=6, Ntau=3, sink="none", material="table1", q_time=W.q_time_paper(6, 1 / 6))
    op = Operator(prob, np.full(prob.Ne, 0.6))
    cm = CoarseMesh(op)
    T = cm.P @ W.rho_uniform(6, 5, 7, 0.0, 1.0)
    TG, _ = cm.G_pri(1, T, 0.0)
    A = (op.C / prob.dtau + op.K)
    b = op.C @ T / prob.dtau + op.load(prob.M * 2)
    r = cm.P.T @ (A @ TG - b)
    assert np.max(np.abs(r)) < 1e-12 * np.max(np.abs(cm.P.T @ b))


def test_coarse_adjoint_step_is_galerkin_orthogonal_on_nested_states():
    prob = make_problem(10, 8, Nt=6, Ntau=3, sink="none", material="table1")
    op = Operator(prob, np.full(prob.Ne, 0.6))
    cm = CoarseMesh(op)
    lam = cm.P @ W.rho_uniform(6, 5, 8, -1.0, 1.0)
    T_hist = np.abs(np.random.default_rng(4).standard_normal((prob.Nt + 1, prob.Nn)))
    lamG, _ = cm.G_adj(1, lam, np.zeros(prob.Ne), T_hist, 0.7)
    from oracle.stepping import adjoint_source_scale
    A = (op.C / prob.dtau + op.K)
    b = op.C @ lam / prob.dtau + adjoint_source_scale(prob, 0.7) * T_hist[prob.M + 1] ** (prob.p - 1)
    r = cm.P.T @ (A @ lamG - b)
    assert np.max(np.abs(r)) < 1e-12 * np.max(np.abs(cm.P.T @ b))


def problem():
    prob = make_problem(10, 8, Nt=12, Ntau=4, dt=1 / 24, material="table1", sink="left_wide",
                        q_time=W.q_time_paper(12, 1 / 24))
    return prob, W.rho_uniform(10, 8, 31, 0.05, 0.95)


def test_oneshot_fixed_point_with_coarse_mesh_G():
    """Warm-started from the exact sequential coarse states of the same design, one one-shot
    pass returns the sequential result whatever G is (Sec. 4.4)."""
    prob, rho = problem()
    op = Operator(prob, rho)
    U, V, seq = coarse_states_from_sequential(op)
    out = oneshot_pass(op, U, V, coarse=CoarseMesh(op))
    assert rel(out["T_hist"], seq["T_hist"]) < 1e-12
    assert abs(out["Theta"] - seq["Theta"]) < 1e-13 * seq["Theta"]
    assert rel(out["grad"], seq["grad"]) < 1e-11


def test_parareal_with_coarse_mesh_G_is_exact_after_Ntau_iterations():
    prob, rho = problem()
    op = Operator(prob, rho)
    seq = sequential_pass(op)
    out = parareal(op, prob.Ntau, coarse=CoarseMesh(op))
    assert rel(out["T_hist"], seq["T_hist"]) < 1e-11
    assert rel(out["grad"], seq["grad"]) < 1e-10
    one = parareal(op, 1, coarse=CoarseMesh(op))
    assert rel(one["grad"], seq["grad"]) > 1e-6          # one iteration is only an estimate


def test_coarse_step_converges_to_the_fine_step_at_second_order():
    """A smooth state on a uniform design: the difference between the coarse-mesh and the
    fine-mesh coarse step falls about fourfold when h halves (both are O(h^2) accurate)."""
    errs = []
    for n in (16, 32):
        prob = make_problem(n, Nt=4, Ntau=2, dt=1 / 16, sink="none")
        op = Operator(prob, np.full(prob.Ne, 0.7))
        x, y = nodes(n, n, prob.h)
        T = np.cos(np.pi * x) * np.cos(np.pi * y) + 1.0
        a, _ = G_pri(op, 0, T, 0.0)
        b, _ = CoarseMesh(op).G_pri(0, T, 0.0)
        errs.append(np.max(np.abs(a - b)))
    assert errs[0] / errs[1] > 3.0, errs


@pytest.mark.parametrize("material", ["simp_k", "table1"])
def test_galerkin_product_of_a_nonuniform_design_is_a_nine_point_stencil_on_2h(material):
    """P^T A P couples each 2h node only to its eight 2h neighbours for any design (the bilinear
    interpolation of a 2h element stays inside it), and it is symmetric positive definite on
    the free 2h nodes: the coarse level of a multigrid cycle stays a 9-point operator."""
    prob = make_problem(10, 8, Nt=4, Ntau=2, sink="left_wide", material=material)
    op = Operator(prob, W.rho_uniform(10, 8, 41, 0.01, 1.0))
    A = (op.C / prob.dtau + op.K).tocsr()
    P = prolongation(prob)
    G = (P.T @ A @ P).tocoo()
    nxH = prob.nx // 2
    iy, ix = np.divmod(G.row, nxH + 1)
    jy, jx = np.divmod(G.col, nxH + 1)
    nz = np.abs(G.data) > 0
    assert np.all(np.abs(iy - jy)[nz] <= 1) and np.all(np.abs(ix - jx)[nz] <= 1)
    Gd = G.toarray()
    free = np.abs(np.diag(Gd)) > 0
    Gf = Gd[np.ix_(free, free)]
    assert np.allclose(Gf, Gf.T, rtol=0, atol=1e-14 * np.max(np.abs(Gf)))
    assert np.min(np.linalg.eigvalsh(Gf)) > 0
