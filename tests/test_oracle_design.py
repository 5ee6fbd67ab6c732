"""Pins of the oracle's design parametrisation and design update (Sec. 2.1, Sec. 3): the
density filter, the threshold projection, their chain rule through the objective, the area
constraint, and the Method of Moving Asymptotes on problems with closed-form optima.  CPU."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from oracle import Operator, sequential_pass
from oracle.design import MMA, Design, filter_matrix, project, project_derivative
from tests.problems import make_problem


def test_filter_rows_average_and_small_radius_is_identity():
    H = filter_matrix(9, 7, 0.1, 0.25)
    assert np.allclose(np.asarray(H.sum(axis=1)).ravel(), 1.0, rtol=0, atol=1e-15)
    assert np.all(H.data > 0)
    I = filter_matrix(9, 7, 0.1, 0.099).toarray()
    assert np.array_equal(I, np.eye(63))


def test_filter_preserves_linear_fields_away_from_the_boundary():
    """The cone weights are symmetric about each centre, so an affine field is reproduced
    wherever the whole disc lies inside the grid."""
    nx, ny, h, r = 20, 16, 0.05, 0.16
    H = filter_matrix(nx, ny, h, r)
    ey, ex = np.divmod(np.arange(nx * ny), nx)
    f = 0.3 + 0.7 * ex - 0.2 * ey
    g = H @ f
    R = int(np.ceil(r / h))
    inner = (ex >= R) & (ex < nx - R) & (ey >= R) & (ey < ny - R)
    assert inner.sum() > 20
    assert np.max(np.abs(g[inner] - f[inner])) < 1e-12
    assert np.max(np.abs(g[~inner] - f[~inner])) > 1e-3      # the boundary rows do differ


def test_projection_fixed_points_limit_and_derivative():
    x = np.linspace(0, 1, 101)
    for beta in (1.0, 8.0, 32.0):
        P = project(x, beta, 0.5)
        assert abs(P[0]) < 1e-15 and abs(P[-1] - 1) < 1e-15 and abs(P[50] - 0.5) < 1e-15
        assert np.all(np.diff(P) > 0)
        eps = 1e-6
        fd = (project(x + eps, beta, 0.5) - project(x - eps, beta, 0.5)) / (2 * eps)
        assert np.max(np.abs(fd - project_derivative(x, beta, 0.5))) < 1e-6 * beta
    assert np.max(np.abs(project(x, 1e-4, 0.3) - x)) < 1e-6       # beta -> 0: the identity


@pytest.mark.parametrize("beta", [2.0, 16.0])
def test_chain_rule_through_filter_projection_and_objective(beta):
    """d Theta(P(H chi)) / d chi and d mean(P(H chi)) / d chi against central differences on every
    element of a small problem with capacity SIMP."""
    nx, ny, Nt = 6, 5, 8
    prob = make_problem(nx, ny, Nt=Nt, dt=0.05, material="table1", sink="left_wide", q_time=W.q_time_paper(Nt, 0.05))
    des = Design(nx, ny, prob.h, 0.35, beta, 0.5)
    chi = W.rho_uniform(nx, ny, 13, 0.3, 0.7)
    rho, dproj = des.forward(chi)
    seq = sequential_pass(Operator(prob, rho))
    g = des.backward(dproj, seq["grad"])
    gv = des.volume_gradient(dproj)
    eps = 1e-6
    fd, fdv = np.zeros_like(g), np.zeros_like(g)
    for e in range(nx * ny):
        cp, cm = chi.copy(), chi.copy()
        cp[e] += eps
        cm[e] -= eps
        rp, rm = des.forward(cp)[0], des.forward(cm)[0]
        fd[e] = (sequential_pass(Operator(prob, rp))["Theta"] - sequential_pass(Operator(prob, rm))["Theta"]) / (2 * eps)
        fdv[e] = (des.volume(rp, 0.3) - des.volume(rm, 0.3)) / (2 * eps)
    assert np.max(np.abs(g - fd)) < 1e-6 * np.max(np.abs(g))
    assert np.max(np.abs(gv - fdv)) < 1e-8 * np.max(np.abs(gv))


def _separable_optimum(c, V, lo, hi):
    """argmin sum c_j / x_j s.t. mean(x) <= V, lo <= x <= hi: x_j = clip(sqrt(c_j / mu)), mean = V."""
    a, b = 1e-12, 1e12
    for _ in range(400):
        mu = np.sqrt(a * b)
        x = np.clip(np.sqrt(c / mu), lo, hi)
        if x.mean() > V:
            a = mu
        else:
            b = mu
    return np.clip(np.sqrt(c / np.sqrt(a * b)), lo, hi)


def test_mma_reaches_the_optimum_of_a_separable_convex_problem():
    rng = np.random.default_rng(3)
    n, V, lo, hi = 200, 0.35, 0.01, 1.0
    c = rng.uniform(0.1, 2.0, n)
    x_star = _separable_optimum(c, V, lo, hi)
    mma = MMA(n, lo, hi, move=0.2)
    x = np.full(n, V)
    for _ in range(150):
        x = mma.update(x, float(np.sum(c / x)), -c / x**2, float(x.mean() - V), np.full(n, 1.0 / n))
    assert np.max(np.abs(x - x_star)) < 1e-5
    assert x.mean() - V < 1e-8


def test_mma_with_an_inactive_constraint_finds_the_box_minimum():
    """min sum (x_j - t_j)^2 with a loose constraint: the minimiser is t clipped to the box."""
    rng = np.random.default_rng(4)
    n = 50
    t = rng.uniform(-0.2, 1.2, n)
    mma = MMA(n, 0.0, 1.0, move=0.3)
    x = np.full(n, 0.5)
    for _ in range(100):
        x = mma.update(x, float(np.sum((x - t) ** 2)), 2 * (x - t), float(x.mean() - 2.0), np.full(n, 1.0 / n))
    assert np.max(np.abs(x - np.clip(t, 0, 1))) < 1e-6
