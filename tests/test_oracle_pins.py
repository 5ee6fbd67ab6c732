"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

None of these compare the oracle with itself: each checks a closed form, an
invariant, a dense brute-force solve, finite differences, or a special case
whose answer is known independently (see the oracle package docstring).
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from oracle import (Operator, element_matrices, objective, oneshot_pass, parareal,
                    sequential_pass, coarse_states_from_sequential)
from oracle.allatonce import adjoint_all_at_once, solve_all_at_once
from oracle.parareal import adjoint_iteration, primal_iteration
from oracle.stepping import sequential_primal
from tests.problems import make_problem


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


# ------------------------------------------------------------------ element level

def test_element_matrices_match_textbook_bilinear_square():
    """Sec. 2.2: Galerkin bilinear square element.  Textbook closed forms:
    K = (1/6)[[4,-1,-2,-1],...] (h-independent in 2D), M = h^2/36 [[4,2,1,2],...], f = h^2/4."""
    for h in (1.0, 0.25, 1.0 / 128):
        Ke, Me, fe = element_matrices(h)
        K_tb = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
        M_tb = np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]]) * h * h / 36.0
        assert np.allclose(Ke, K_tb, rtol=0, atol=1e-14)
        assert np.allclose(Me, M_tb, rtol=1e-13, atol=0)
        assert np.allclose(fe, h * h / 4, rtol=1e-13)
        assert np.allclose(Ke.sum(axis=1), 0, atol=1e-14)       # constants are in the kernel
        assert abs(Me.sum() - h * h) < 1e-14                     # total mass = area


# ------------------------------------------------------------------ closed-form decay

def _mu1(m, n, h):
    th = m * np.pi / n
    return 6.0 / h ** 2 * (1 - np.cos(th)) / (2 + np.cos(th))


@pytest.mark.parametrize("nx,ny,mx,my", [(6, 6, 1, 0), (8, 5, 2, 1), (7, 9, 3, 3), (12, 12, 4, 2)])
def test_separable_eigenmode_decays_in_closed_form(nx, ny, mx, my):
    """Uniform design, all-Neumann edges, q = 0: the nodal field cos(mx pi x/Lx) cos(my pi y/Ly)
    is an eigenvector of K v = mu C v with mu = (k/c)(mu1(mx) + mu1(my)), mu1(m) =
    (6/h^2)(1 - cos(m pi/n))/(2 + cos(m pi/n)), so backward Euler (Eq. 2.7) gives
    T_j = (1 + dt mu)^-j T_0 exactly.  A non-square grid catches x/y transpositions."""
    h = 1.0 / max(nx, ny)
    Nt, dt = 7, 0.013
    x = np.arange(nx + 1) * h
    y = np.arange(ny + 1) * h
    T0 = (np.cos(my * np.pi * y / (ny * h))[:, None] * np.cos(mx * np.pi * x / (nx * h))[None, :]).reshape(-1)
    prob = make_problem(nx, ny, Nt=Nt, dt=dt, sink="none", material="table1", q_time=np.zeros(Nt + 1), T0=T0, h=h)
    rho = np.full(nx * ny, 0.7)
    op = Operator(prob, rho)
    T_hist, theta = sequential_primal(op)
    mat = prob.material
    k = mat.kmin + (mat.k0 - mat.kmin) * 0.7 ** mat.pk
    c = mat.cmin + (mat.c0 - mat.cmin) * 0.7 ** mat.pc
    mu = (k / c) * (_mu1(mx, nx, h) + _mu1(my, ny, h))
    for j in range(Nt + 1):
        assert rel(T_hist[j], T0 * (1 + dt * mu) ** (-j)) < 1e-10   # round-off grows as the mode decays
    # the objective of Eq. 2.11 of this history, in closed form
    s = sum(np.sum(T0 ** prob.p) * (1 + dt * mu) ** (-j * prob.p) for j in range(1, Nt + 1))
    assert abs(theta[-1] - (s / (Nt * prob.Ne)) ** (1 / prob.p)) < 1e-13 * theta[-1]


def test_eigenmode_approaches_continuous_decay():
    """The continuous mode decays as exp(-pi^2 (mx^2/Lx^2 + my^2/Ly^2) k t / c); the discrete
    decay converges to it as h, dt -> 0 (first order in dt)."""
    errs = []
    for n, Nt in ((8, 10), (16, 20), (32, 40)):
        h = 1.0 / n
        x = np.arange(n + 1) * h
        T0 = (np.cos(np.pi * x)[:, None] * np.ones(n + 1)[None, :]).reshape(-1)  # mode (0, 1)
        prob = make_problem(n, Nt=Nt, dt=0.05 / Nt, sink="none", q_time=np.zeros(Nt + 1), T0=T0)
        op = Operator(prob, np.full(n * n, 1.0))
        T_hist, _ = sequential_primal(op)
        exact = np.exp(-np.pi ** 2 * 1.0 * 0.05)
        errs.append(abs(T_hist[-1][0] / T0[0] - exact))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.6 * errs[1]


# ------------------------------------------------------------------ conservation

def test_discrete_energy_balance():
    """Summing Eq. 2.7 over the free nodes and using K 1 = 0 gives
    1^T C_ff (T_j - T_{j-1}) = dt (1^T q_f + sum_{d in D} (K T_j)_d): the heat stored equals the
    heat supplied plus the (negative) reaction at the sink.  Also pins the load total:
    the unit load sums to the domain area."""
    prob = make_problem(10, 7, Nt=9, dt=0.02, material="table1", sink="left_wide",
                        q_time=W.q_time_paper(9, 0.02))
    rho = W.rho_uniform(10, 7, 5, 0.0, 1.0)
    op = Operator(prob, rho)
    assert abs(op.f.sum() - 10 * 7 * prob.h ** 2) < 1e-14
    assert np.max(np.abs(op.K @ np.ones(prob.Nn))) < 1e-14
    T_hist, _ = sequential_primal(op)
    f = op.free
    D = ~f
    for j in range(1, prob.Nt + 1):
        lhs = np.sum((op.C @ (T_hist[j] - T_hist[j - 1]))[f])
        rhs = prob.dt * (np.sum(op.load(j)[f]) + np.sum((op.K @ T_hist[j])[D]))
        assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1e-3)


def test_zero_at_dirichlet_nodes_and_positive_interior():
    prob = make_problem(8, Nt=5, dt=0.05)
    op = Operator(prob, W.rho_plain(8, 8, 0))
    T_hist, _ = sequential_primal(op)
    assert np.all(T_hist[:, ~op.free] == 0)
    assert np.all(T_hist[1:, op.free] > 0)


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("material", ["simp_k", "table1"])
def test_dense_all_at_once_matches_sequential(material):
    """Eq. 2.8-2.9 (M S = Q) and Eq. 4.3-4.5 (M^T Lambda = Nt dTheta/dS^T, grad = -Lambda^T dR/drho / Nt)
    solved densely on a 4x3 grid reproduce the sequential primal, objective, adjoint and gradient."""
    Nt = 6
    prob = make_problem(4, 3, Nt=Nt, dt=0.07, material=material, sink="left_wide",
                        q_time=W.q_time_paper(Nt, 0.07), p=8.0)
    rho = W.rho_uniform(4, 3, 2, 0.1, 0.9)
    op = Operator(prob, rho)
    seq = sequential_pass(op)
    T_dense, Mbig = solve_all_at_once(op)
    assert rel(seq["T_hist"], T_dense) < 1e-13
    lam, grad, Theta = adjoint_all_at_once(op, T_dense, Mbig)
    assert abs(seq["Theta"] - Theta) < 1e-14 * Theta
    assert abs(objective(seq["T_hist"], prob) - Theta) < 1e-14 * Theta
    assert rel(seq["lam"][1:Nt + 1], lam[1:Nt + 1]) < 1e-12
    assert rel(seq["grad"], grad) < 1e-12


# ------------------------------------------------------------------ finite differences

@pytest.mark.parametrize("material,p", [("table1", 8.0), ("table1", 20.0), ("simp_k", 8.0)])
def test_gradient_matches_central_differences(material, p):
    """The discrete adjoint (Sec. 4.1) is exact for the sequential solution, so it must match
    central differences (eps = 1e-6) of Theta on every element to FD truncation/round-off."""
    nx, ny, Nt = 5, 4, 8
    prob = make_problem(nx, ny, Nt=Nt, dt=0.06, material=material, sink="left_wide", p=p,
                        q_time=W.q_time_paper(Nt, 0.06))
    rho = W.rho_uniform(nx, ny, 7, 0.15, 0.85)
    g = sequential_pass(Operator(prob, rho))["grad"]
    eps = 1e-6
    fd = np.zeros_like(g)
    for e in range(prob.Ne):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += eps
        rm[e] -= eps
        fd[e] = (sequential_pass(Operator(prob, rp))["Theta"] - sequential_pass(Operator(prob, rm))["Theta"]) / (2 * eps)
    assert rel(g, fd) < 1e-6


def test_gradient_fd_on_plain32_sample():
    """32x32, 100 steps (the plain FP64 workload): central differences on 32 random elements."""
    w = W.workload("plain32")
    prob = make_problem(32, Nt=w["Nt"], dt=w["dt"], p=w["p"])
    rho = W.rho_plain(32, 32, 0)
    g = sequential_pass(Operator(prob, rho))["grad"]
    eps = 1e-6
    for e in W.fd_elements(prob.Ne, 32, seed=3):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += eps
        rm[e] -= eps
        fd = (sequential_pass(Operator(prob, rp))["Theta"] - sequential_pass(Operator(prob, rm))["Theta"]) / (2 * eps)
        assert abs(fd - g[e]) < 1e-6 * np.max(np.abs(g))


# ------------------------------------------------------------------ Parareal

@pytest.mark.parametrize("Nt,Ntau", [(12, 3), (12, 4), (10, 5)])
def test_parareal_exact_after_Ntau_iterations(Nt, Ntau):
    """Sec. 4.2: after as many iterations as slices, Parareal reproduces the sequential fine
    solution; the modified history, Theta and the reverse adjoint gradient follow."""
    prob = make_problem(6, 5, Nt=Nt, Ntau=Ntau, dt=0.5 / Nt, material="table1", sink="left_wide",
                        q_time=W.q_time_paper(Nt, 0.5 / Nt))
    op = Operator(prob, W.rho_uniform(6, 5, 11, 0.1, 0.9))
    seq = sequential_pass(op)
    par = parareal(op, Ntau)
    assert rel(par["T_hist"], seq["T_hist"]) < 1e-12
    assert abs(par["Theta"] - seq["Theta"]) < 1e-13 * seq["Theta"]
    assert rel(par["grad"], seq["grad"]) < 1e-11
    # and fewer iterations are not exact (the test would be vacuous otherwise)
    assert rel(parareal(op, 1)["grad"], seq["grad"]) > 1e-6


@pytest.mark.parametrize("Nt,Ntau", [(6, 6), (6, 1)])
def test_degenerate_M1_and_single_slice_are_exact_in_one_iteration(Nt, Ntau):
    """M = 1 makes G equal to F; N_tau = 1 makes F the whole sequential run.  Either way one
    Parareal iteration is exact."""
    prob = make_problem(5, Nt=Nt, Ntau=Ntau, dt=0.1, material="table1", sink="left_wide")
    op = Operator(prob, W.rho_uniform(5, 5, 4, 0.1, 0.9))
    seq = sequential_pass(op)
    par = parareal(op, 1)
    assert rel(par["T_hist"], seq["T_hist"]) < 1e-12
    assert rel(par["grad"], seq["grad"]) < 1e-11


def test_fig1_indexing_Nt15_Ntau3():
    """Fig. 1: Nt = 15, Ntau = 3, M = 5, coarse points t_0, t_5, t_10, t_15.  Slice s writes the
    history rows 5s+1..5s+5; v_n = (lambda_{5n+1}, g_{5n+1}), v_3 = 0 and v_0 holds g_1 = grad."""
    prob = make_problem(4, Nt=15, Ntau=3, dt=0.02, sink="left_wide")
    assert prob.M == 5
    op = Operator(prob, W.rho_uniform(4, 4, 1, 0.2, 0.8))
    (U_T, U_th), (V_l, V_g), seq = coarse_states_from_sequential(op)
    assert np.array_equal(U_T, seq["T_hist"][[0, 5, 10, 15]])
    assert np.array_equal(U_th, seq["theta"][[0, 5, 10, 15]])
    assert np.array_equal(V_l, seq["lam"][[1, 6, 11, 16]])
    assert np.all(V_l[3] == 0) and np.all(V_g[3] == 0)
    assert np.array_equal(V_g[0], seq["grad"])
    # the forward iteration writes slice s's uncorrected intermediates into rows 5s+1..5s+4 and
    # the corrected coarse state into row 5s+5 (Sec. 4.3).  Perturb the guess for u_1 only: slice 1's
    # intermediates (6..9) and the corrected t_10 move, t_15 moves through G(u_2^new), while slice
    # 2's intermediates (11..14) come from F(u_2^old), which is unperturbed, and stay put.
    U_T2 = U_T.copy()
    U_T2[1] *= 1.5
    out = primal_iteration(op, (U_T2, U_th))
    moved = [j for j in range(16) if not np.allclose(out["T_hist"][j], seq["T_hist"][j], rtol=1e-12, atol=0)]
    assert moved == [6, 7, 8, 9, 10, 15]


def _coarsened(prob, q_time):
    """The problem the coarse propagator steps when the substitution of Sec. 4.4 (dt -> dtau,
    Nt -> Ntau, n -+ 1 -> n -+ M) is applied to Alg. 1-2: Ntau backward-Euler steps of size
    dtau whose loads sit at the coarse points t_{Ms}."""
    Ntau = prob.Ntau
    return make_problem(prob.nx, prob.ny, Nt=Ntau, Ntau=Ntau, dt=prob.dtau, p=prob.p,
                        material=prob.material, sink=np.asarray(prob.dirichlet), h=prob.h,
                        q_time=np.asarray(q_time)[::prob.M].copy(), T0=prob.T0)


@pytest.mark.parametrize("M,Ntau", [(3, 4), (5, 3)])
def test_coarse_primal_propagator_chained_is_sequential_stepping_of_the_coarsened_problem(M, Ntau):
    """G_pri (Sec. 4.4) chained from u_0 over every slice is backward Euler with step dtau = M dt
    and the load at the new coarse point, and its theta accumulates with the divisor Ntau Ne.
    That is the sequential primal pass (Alg. 1, Eq. 2.7, Eq. 2.11) of the problem with Ntau
    steps of size dtau and the loads q(t_{Ms}), computed here by the plain sequential stepper.
    The paper's time-varying load (Eq. 5.1) and capacity SIMP (Table 1) make a wrong load
    index or a wrong divisor visible."""
    from oracle.parareal import G_pri
    Nt = M * Ntau
    dt = 0.6 / Nt
    qt = W.q_time_paper(Nt, dt)
    prob = make_problem(7, 5, Nt=Nt, Ntau=Ntau, dt=dt, material="table1", sink="left_wide", q_time=qt)
    op = Operator(prob, W.rho_uniform(7, 5, 21, 0.1, 0.9))
    cprob = _coarsened(prob, qt)
    Tc, thc = sequential_primal(Operator(cprob, op.rho))
    T, th = np.zeros(prob.Nn), 0.0
    for s in range(Ntau):
        T, th = G_pri(op, s, T, th)
        assert rel(T, Tc[s + 1]) < 1e-13
        assert abs(th - thc[s + 1]) <= 1e-13 * thc[s + 1]
    # the pin is not vacuous: the coarse chain differs from the fine run at the same times
    T_fine, _ = sequential_primal(op)
    assert rel(T_fine[Nt], Tc[Ntau]) > 1e-4


@pytest.mark.parametrize("M,Ntau", [(3, 4), (5, 3)])
def test_coarse_adjoint_propagator_chained_is_sequential_adjoint_of_the_coarsened_problem(M, Ntau):
    """G_adj (Sec. 4.4) solves for lambda_k, k = Ms+1, from lambda_{k+M} with the source at T_k,
    and adds to g the Eq. 4.7 bracket of (T_k - T_{k-M})/dtau with the divisor Ntau (T_{k-M}
    read as T_0 for s = 0).  Given a history whose rows Ms+1 hold the coarsened problem's
    temperatures T'_{s+1} and whose row 0 holds T_0, the chain from v_Ntau = 0 must be the
    sequential discrete adjoint (Alg. 2) of the coarsened problem: lambda'_{s+1} and g'_{s+1}.
    Every other history row holds noise, so reading a wrong row fails, and the capacity SIMP
    of Table 1 makes the T_{k-M} term count."""
    from oracle.parareal import G_adj
    from oracle.stepping import sequential_adjoint
    Nt = M * Ntau
    dt = 0.6 / Nt
    qt = W.q_time_paper(Nt, dt)
    rng = np.random.default_rng(8)
    T0 = rng.uniform(0.0, 0.3, (7 + 1) * (5 + 1))
    prob = make_problem(7, 5, Nt=Nt, Ntau=Ntau, dt=dt, material="table1", sink="left_wide", q_time=qt, T0=T0)
    prob.T0[np.asarray(prob.dirichlet, bool)] = 0.0
    op = Operator(prob, W.rho_uniform(7, 5, 22, 0.1, 0.9))
    cprob = _coarsened(prob, qt)
    cop = Operator(cprob, op.rho)
    Tc, thc = sequential_primal(cop)
    Theta = thc[-1]
    lam_c, g_c = sequential_adjoint(cop, Tc, Theta)
    T_hist = rng.uniform(1.0, 2.0, (Nt + 1, prob.Nn))
    T_hist[0] = Tc[0]
    for s in range(Ntau):
        T_hist[M * s + 1] = Tc[s + 1]
    lam, g = np.zeros(prob.Nn), np.zeros(prob.Ne)
    for s in range(Ntau - 1, -1, -1):
        lam, g = G_adj(op, s, lam, g, T_hist, Theta)
        assert rel(lam, lam_c[s + 1]) < 1e-12
        assert rel(g, g_c[s + 1]) < 1e-11
    # the dC/drho term is present: with unit capacity the gradient changes
    assert np.max(np.abs(op.dc)) > 0


def test_oneshot_fixed_point():
    """Alg. 3 warm start from the exact sequential coarse states of the same design returns the
    sequential history, objective and gradient (G(u^new) and G(u^old) cancel exactly)."""
    prob = make_problem(8, 6, Nt=24, Ntau=4, dt=1 / 24, material="table1", sink="left_wide",
                        q_time=W.q_time_paper(24, 1 / 24))
    op = Operator(prob, W.rho_uniform(8, 6, 9, 0.1, 0.9))
    U, V, seq = coarse_states_from_sequential(op)
    out = oneshot_pass(op, U, V)
    assert rel(out["T_hist"], seq["T_hist"]) < 1e-13
    assert abs(out["Theta"] - seq["Theta"]) < 1e-14 * seq["Theta"]
    assert rel(out["grad"], seq["grad"]) < 1e-12


def test_oneshot_error_shrinks_with_design_change():
    """With the warm start taken from a nearby design, the one-shot estimate's error against the
    sequential result of the current design shrinks (about linearly) with the design change."""
    prob = make_problem(8, Nt=32, Ntau=8, dt=1 / 32, sink="left")
    rho = W.rho_uniform(8, 8, 2, 0.2, 0.8)
    op = Operator(prob, rho)
    seq = sequential_pass(op)
    errs = []
    for amp in (1e-1, 1e-2, 1e-3):
        rho_old = W.rho_warm_perturb(rho, seed=5, amp=amp)
        U, V, _ = coarse_states_from_sequential(Operator(prob, rho_old))
        out = oneshot_pass(op, U, V)
        errs.append(np.linalg.norm(out["grad"] - seq["grad"]) / np.linalg.norm(seq["grad"]))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.05 * errs[0]


def test_adjoint_correction_independent_of_carried_g():
    """Reading of Eq. 4.14 on v = (lambda, g): g enters F_adj and G_adj additively, so g^old
    cancels in F(v^old) - G(v^old); the slice-local increment form is equivalent."""
    prob = make_problem(6, Nt=12, Ntau=3, dt=1 / 12, material="table1", sink="left_wide")
    op = Operator(prob, W.rho_uniform(6, 6, 3, 0.1, 0.9))
    U, V, seq = coarse_states_from_sequential(op)
    pri = primal_iteration(op, U)
    a = adjoint_iteration(op, V, pri["T_hist"], pri["Theta"])
    b = adjoint_iteration(op, (V[0], np.zeros_like(V[1])), pri["T_hist"], pri["Theta"])
    assert rel(a["V"][1], b["V"][1]) < 1e-12


@pytest.mark.parametrize("prop", ["F_adj", "G_adj"])
def test_adjoint_propagators_are_affine_in_the_state_and_linear_in_the_source_scale(prop):
    """lambda solves (C/dt + K) lambda_j = C/dt lambda_{j+1} + c T_j^(p-1) with c = Theta^(1-p)/Ne
    (Eq. 4.6), and g accumulates a term linear in lambda (Eq. 4.7).  So F_adj and G_adj split
    into a part driven by the state and a part proportional to c: their difference for two
    objectives does not depend on the state, and the state-free part scales with c."""
    from oracle.parareal import F_adj, G_adj
    prob = make_problem(8, 6, Nt=12, Ntau=3, dt=1 / 12, material="table1", sink="left_wide")
    op = Operator(prob, W.rho_uniform(8, 6, 5, 0.1, 0.9))
    T_hist, _ = sequential_primal(op)
    rng = np.random.default_rng(11)
    lam = rng.standard_normal(prob.Nn)
    lam[np.asarray(prob.dirichlet, bool)] = 0.0
    g = rng.standard_normal(prob.Ne)
    zl, zg = np.zeros(prob.Nn), np.zeros(prob.Ne)
    fn = F_adj if prop == "F_adj" else G_adj
    s = 1
    Th1, Th2 = 0.7, 1.3
    c1, c2 = Th1 ** (1 - prob.p), Th2 ** (1 - prob.p)
    a1 = fn(op, s, lam, g, T_hist, Th1)
    a2 = fn(op, s, lam, g, T_hist, Th2)
    z1 = fn(op, s, zl, zg, T_hist, Th1)
    z2 = fn(op, s, zl, zg, T_hist, Th2)
    for i in range(2):
        # the state-driven part cancels in the difference of two objectives
        assert rel(a1[i] - a2[i], z1[i] - z2[i]) < 1e-10
        # the state-free part is proportional to c
        assert rel(z2[i], (c2 / c1) * z1[i]) < 1e-12


# ------------------------------------------------------------------ symmetry, objective identities

def test_mirror_symmetry_about_mid_height():
    """A design and sink symmetric about y = L/2 give a temperature and gradient with the same symmetry."""
    n = 10
    prob = make_problem(n, Nt=10, dt=0.02, sink="left")
    rho = W.rho_mirror_y(n, n, 8)
    seq = sequential_pass(Operator(prob, rho))
    T = seq["T_hist"].reshape(-1, n + 1, n + 1)
    assert np.max(np.abs(T - T[:, ::-1, :])) < 1e-12 * np.max(np.abs(T))
    g = seq["grad"].reshape(n, n)
    assert np.max(np.abs(g - g[::-1, :])) < 1e-10 * np.max(np.abs(g))


def test_objective_of_constant_field():
    """Eq. 2.11 with T_j = a at every node and step: Theta = a (Nn/Ne)^(1/p)."""
    prob = make_problem(6, 4, Nt=5, p=8.0)
    a = 0.37
    T_hist = np.full((prob.Nt + 1, prob.Nn), a)
    assert abs(objective(T_hist, prob) - a * (prob.Nn / prob.Ne) ** (1 / 8)) < 1e-15


def test_theta_and_gradient_are_homogeneous_in_the_load():
    """T is linear in q and the power mean is 1-homogeneous, so Theta and grad scale with q."""
    prob1 = make_problem(6, Nt=6, dt=0.05, material="table1")
    prob3 = make_problem(6, Nt=6, dt=0.05, material="table1", q_elem=np.full(36, 3.0))
    rho = W.rho_uniform(6, 6, 1, 0.1, 0.9)
    s1 = sequential_pass(Operator(prob1, rho))
    s3 = sequential_pass(Operator(prob3, rho))
    assert abs(s3["Theta"] - 3 * s1["Theta"]) < 1e-13 * s3["Theta"]
    assert rel(s3["grad"], 3 * s1["grad"]) < 1e-12


def test_dirichlet_node_counts():
    """Centred 10% of the left edge, inclusive: 3 / 7 / 9 / 13 / 19 / 25 / 51 nodes for
    n = 32 / 64 / 96 / 128 / 192 / 256 / 512."""
    for n, cnt in ((32, 3), (64, 7), (96, 9), (128, 13), (192, 19), (256, 25), (512, 51)):
        assert int(W.dirichlet_left_centre(n, n, 1.0 / n).sum()) == cnt


def test_batch48_composition():
    """The 48-design batching workload: sizes cycled by index mod 5 (10 x 64^2, 10 x 96^2,
    10 x 128^2, 9 x 192^2, 9 x 256^2), (Nt, Ntau) by index mod 3 over (512, 16), (1024, 32),
    (2048, 64) (M = 32 throughout), conductivity SIMP, p = 8, rho ~ U(0.2, 0.8) with seed 100 + index."""
    ds = W.batch48()
    assert len(ds) == 48 and [d["index"] for d in ds] == list(range(48))
    sizes = [d["n"] for d in ds]
    assert {n: sizes.count(n) for n in set(sizes)} == {64: 10, 96: 10, 128: 10, 192: 9, 256: 9}
    for i, d in enumerate(ds):
        assert d["n"] == (64, 96, 128, 192, 256)[i % 5]
        assert (d["Nt"], d["Ntau"]) == ((512, 16), (1024, 32), (2048, 64))[i % 3]
        assert d["Nt"] // d["Ntau"] == 32 and d["dt"] == 1.0 / d["Nt"] and d["p"] == 8.0
        assert d["material"] == "simp_k" and d["seed"] == 100 + i
        rho = d["rho"]
        assert rho.shape == (d["n"] * d["n"],) and rho.min() >= 0.2 and rho.max() <= 0.8
        assert np.array_equal(rho, np.random.default_rng(100 + i).uniform(0.2, 0.8, d["n"] * d["n"]))


def test_sparse_lu_and_band_cholesky_give_the_same_passes():
    """The oracle factors C/dt + K by banded Cholesky on narrow grids and by sparse LU on wide
    ones (the band factor of a 512 x 512 grid takes minutes).  Both are direct solves of the
    same systems, so the sequential pass and the one-shot pass agree to rounding."""
    prob = make_problem(24, 18, Nt=12, Ntau=3, dt=0.4 / 12, material="table1", sink="left_wide",
                        q_time=W.q_time_paper(12, 0.4 / 12))
    rho = W.rho_uniform(24, 18, 41, 0.05, 0.95)
    out = {}
    for solver in ("band", "lu"):
        op = Operator(prob, rho, solver=solver)
        assert op._factor(prob.dt)[0] == solver
        U, V, seq = coarse_states_from_sequential(Operator(prob, W.rho_warm_perturb(rho, seed=42, amp=0.05),
                                                           solver=solver))
        out[solver] = (sequential_pass(op), oneshot_pass(op, U, V))
    (sb, ob), (sl, ol) = out["band"], out["lu"]
    assert rel(sl["T_hist"], sb["T_hist"]) < 1e-13 and rel(sl["grad"], sb["grad"]) < 1e-12
    assert rel(ol["T_hist"], ob["T_hist"]) < 1e-13 and rel(ol["grad"], ob["grad"]) < 1e-12
    # the automatic choice switches at the band width
    from oracle.stepping import BAND_MAX
    wide = make_problem(BAND_MAX + 1, 4, Nt=2, dt=0.1)
    assert Operator(wide, np.full(wide.Ne, 0.5))._factor(0.1)[0] == "lu"
    assert Operator(prob, rho)._factor(prob.dt)[0] == "band"
