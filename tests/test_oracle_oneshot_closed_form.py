"""Pin of the one-shot pass for a design that differs from the warm-start design (Sec. 4.4, the
iteration body of Alg. 3), against closed forms on a problem that reduces to scalars.

Setting: Dirichlet sinks on the whole boundary, no load, uniform designs, and an initial state
v = sin(mx pi x / Lx) sin(my pi y / Ly).  On the free (interior) nodes v is an eigenvector of
both the capacity and the conduction matrices of the Q1 elements (Sec. 2.2): C v = c mh v and
K v = k kh v with mh = m1x m1y and kh = kx m1y + m1x ky, where m1 = h (2 + cos t) / 3 and
k1 = 2 (1 - cos t) / h are the 1D mass and stiffness eigenvalues of the mode (t = m pi / n).
So every backward-Euler step (Eq. 2.7) maps a multiple of v to a multiple of v.  With the
modified objective of Sec. 7.1 at p = 2, the adjoint source 2 T / Ne (Eq. 4.6 with Theta~) is
a multiple of v too, and every adjoint state stays a multiple of v.

The warm start is the exact sequential solution of the old design rho_a (written in closed form
here, not taken from the oracle).  The pass runs with the current design rho_b.  Then:
  * T at the coarse points: beta_{n+1} = R beta_n + (r^M - R) A^n, so
    beta_n = R^n + (r^M - R)(R^n - A^n)/(R - A), with r = 1/(1 + dt mu_b),
    R = 1/(1 + dtau mu_b), A = (1/(1 + dt mu_a))^M and mu = (k/c)(kh/mh).
  * T between the coarse points: the uncorrected F intermediates r^i A^s (Sec. 4.3).
  * Theta~: an explicit sum over the slices of the G(new), F(old) and G(old) increments.
  * lambda and the gradient: explicit sums over each slice's fine steps and its coarse step.
    The gradient of element e is a combination of the element's quadratic forms
    v_e^T Ke v_e and v_e^T Me v_e of the textbook matrices, with the current design's dk and dc.
  * The old g states cancel out of the corrections (F_g - G_g holds no g_old), so the gradient
    does not depend on them.
A dropped or mis-indexed term in the oracle's vector code (a time index, the slice bounds of the
history, the divisor of a coarse increment, the T rows a coarse adjoint step reads, the step of
a coarse propagator, a correction without its G(old) term) moves one of these values; the last
tests plant such mistakes in the oracle and see them fail.  The load is zero here: its indexing
is pinned by the coarse propagators' pin at M > 1 (G_pri chained equals the coarsened problem)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import Operator, oneshot_pass
from tests.problems import make_problem

KE = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
ME1 = np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]]) / 36.0   # times h^2


def _setup(nx, ny, mx, my, Nt, Ntau, p, dt, rho_a, rho_b, modified=True):
    h = 1.0 / max(nx, ny)
    x = np.arange(nx + 1) * h
    y = np.arange(ny + 1) * h
    v = (np.sin(my * np.pi * y / (ny * h))[:, None] * np.sin(mx * np.pi * x / (nx * h))[None, :]).reshape(-1)
    sink = np.zeros((ny + 1, nx + 1), dtype=bool)
    sink[0, :] = sink[-1, :] = sink[:, 0] = sink[:, -1] = True
    v[sink.reshape(-1)] = 0.0
    prob = make_problem(nx, ny, Nt=Nt, Ntau=Ntau, dt=dt, p=p, material="table1", sink=sink.reshape(-1),
                        q_time=np.zeros(Nt + 1), T0=v, h=h, modified_objective=modified)
    mat = prob.material
    k = lambda r: mat.kmin + (mat.k0 - mat.kmin) * r ** mat.pk
    c = lambda r: mat.cmin + (mat.c0 - mat.cmin) * r ** mat.pc
    tx, ty = mx * np.pi / nx, my * np.pi / ny
    m1x, m1y = h * (2 + np.cos(tx)) / 3, h * (2 + np.cos(ty)) / 3
    k1x, k1y = 2 * (1 - np.cos(tx)) / h, 2 * (1 - np.cos(ty)) / h
    S = dict(h=h, v=v, prob=prob, mh=m1x * m1y, kh=k1x * m1y + m1x * k1y, modified=modified,
             ka=k(rho_a), ca=c(rho_a), kb=k(rho_b), cb=c(rho_b),
             dkb=mat.pk * (mat.k0 - mat.kmin) * rho_b ** (mat.pk - 1),
             dcb=mat.pc * (mat.c0 - mat.cmin) * rho_b ** (mat.pc - 1))
    return S


def _closed_form(S, Nt, Ntau, p, dt):
    """Amplitudes of T_hist, Theta~, the lambda amplitudes at the coarse points and the two
    coefficients (of v_e^T Ke v_e and v_e^T Me v_e) of the gradient."""
    prob = S["prob"]
    M = Nt // Ntau
    dtau = M * dt
    Ne = prob.Ne
    Pp = float(np.sum(np.abs(S["v"]) ** p))
    mu_a = S["ka"] * S["kh"] / (S["ca"] * S["mh"])
    mu_b = S["kb"] * S["kh"] / (S["cb"] * S["mh"])
    ra, r, R = 1 / (1 + dt * mu_a), 1 / (1 + dt * mu_b), 1 / (1 + dtau * mu_b)
    A = ra ** M
    alpha = np.array([A ** s for s in range(Ntau + 1)])                    # old coarse states
    beta = np.array([R ** n + (r ** M - R) * (R ** n - A ** n) / (R - A) for n in range(Ntau + 1)])
    tau = np.zeros(Nt + 1)                                                  # T_hist amplitudes
    tau[0] = 1.0
    for s in range(Ntau):
        for i in range(1, M):
            tau[M * s + i] = r ** i * alpha[s]
        tau[M * (s + 1)] = beta[s + 1]
    if S["modified"]:
        # Theta~ (plain sum of Sec. 7.1): G(new) + F(old) - G(old) increments of every slice
        Theta = sum(Pp / Ne * ((R * beta[s]) ** p / Ntau
                               + sum((r ** i * alpha[s]) ** p for i in range(1, M + 1)) / Nt
                               - (R * alpha[s]) ** p / Ntau) for s in range(Ntau))
        Theta_a = None
    else:
        # the power mean of Eq. 2.11 carried as theta itself (Sec. 4.4): each propagator adds
        # its increment under the p-th power, the correction acts on theta
        th_old = [(sum(ra ** (p * j) for j in range(1, M * s + 1)) * Pp / (Nt * Ne)) ** (1 / p)
                  for s in range(Ntau + 1)]
        thG = lambda th, amp: (th ** p + (R * amp) ** p * Pp / (Ntau * Ne)) ** (1 / p)
        th = 0.0
        for s in range(Ntau):
            thF = (th_old[s] ** p + sum((r ** i * alpha[s]) ** p for i in range(1, M + 1)) * Pp / (Nt * Ne)) ** (1 / p)
            th = thG(th, beta[s]) + thF - thG(th_old[s], alpha[s])
        Theta, Theta_a = th, th_old[Ntau]
    if p != 2:
        return dict(tau=tau, Theta=Theta)
    # adjoint source scale: p / Ne (Sec. 7.1), or Theta^(1-p) / Ne (Eq. 4.6) with the pass's
    # corrected Theta (and the old design's exact Theta for its sequential adjoint)
    sig = 2.0 / Ne if S["modified"] else Theta ** (1 - p) / Ne
    sig_a = 2.0 / Ne if S["modified"] else Theta_a ** (1 - p) / Ne
    # old adjoint (exact sequential, design a): lambda_j = sum_{i >= j} ra^(i-j+1) dt sig ra^i / (ca mh)
    lam_a = np.zeros(Nt + 2)
    for j in range(1, Nt + 1):
        lam_a[j] = sum(ra ** (i - j + 1) * dt * sig_a * ra ** i / (S["ca"] * S["mh"]) for i in range(j, Nt + 1))
    lam_old = np.array([lam_a[M * n + 1] if n < Ntau else 0.0 for n in range(Ntau + 1)])
    cb_mh = S["cb"] * S["mh"]

    def fine(s, x):
        """F_adj over slice s from amplitude x: the amplitude at every fine step j (after the
        step) and the two gradient coefficients it adds (with the -1/Nt of Eq. 4.7)."""
        top = M * (s + 1)
        lam = {j: r ** (top + 1 - j) * x + sum(r ** (i - j + 1) * dt * sig * tau[i] / cb_mh for i in range(j, top + 1))
               for j in range(M * s + 1, top + 1)}
        ck = -sum(lam[j] * S["dkb"] * tau[j] for j in lam) / Nt
        cm = -sum(lam[j] * S["dcb"] * (tau[j] - tau[j - 1]) / dt for j in lam) / Nt
        return lam[M * s + 1], ck, cm

    def coarse(s, x):
        """G_adj over slice s: one step of dtau solving for lambda_k, k = M s + 1, from T_k and
        T_{k-M} (T_0 for s = 0)."""
        kk, kp = M * s + 1, max(M * s + 1 - M, 0)
        lam = R * x + R * dtau * sig * tau[kk] / cb_mh
        return lam, -lam * S["dkb"] * tau[kk] / Ntau, -lam * S["dcb"] * (tau[kk] - tau[kp]) / dtau / Ntau

    lam_new = np.zeros(Ntau + 1)
    gk = gm = 0.0                                        # gradient coefficients, g_Ntau = 0
    for s in range(Ntau - 1, -1, -1):
        lG_new, kG_new, mG_new = coarse(s, lam_new[s + 1])
        lF_old, kF_old, mF_old = fine(s, lam_old[s + 1])
        lG_old, kG_old, mG_old = coarse(s, lam_old[s + 1])
        lam_new[s] = lG_new + lF_old - lG_old
        gk, gm = gk + kG_new + kF_old - kG_old, gm + mG_new + mF_old - mG_old
    return dict(tau=tau, Theta=Theta, lam_old=lam_old, lam_new=lam_new, gk=gk, gm=gm)


def _element_forms(S):
    prob = S["prob"]
    nx, ny, h, v = prob.nx, prob.ny, S["h"], S["v"]
    qk, qm = np.zeros(nx * ny), np.zeros(nx * ny)
    for ey in range(ny):
        for ex in range(nx):
            n0 = ey * (nx + 1) + ex
            ve = v[[n0, n0 + 1, n0 + nx + 2, n0 + nx + 1]]          # counter-clockwise
            qk[ey * nx + ex] = ve @ KE @ ve
            qm[ey * nx + ex] = h * h * (ve @ ME1 @ ve)
    return qk, qm


def _old_states(S, Nt, Ntau, p, dt, lam_old, rng):
    """The warm start: exact sequential coarse states of design a (closed form), g arbitrary."""
    prob = S["prob"]
    M = Nt // Ntau
    mu_a = S["ka"] * S["kh"] / (S["ca"] * S["mh"])
    ra = 1 / (1 + dt * mu_a)
    Pp = float(np.sum(np.abs(S["v"]) ** p))
    U_T = np.array([ra ** (M * s) * S["v"] for s in range(Ntau + 1)])
    U_th = np.array([sum(ra ** (p * j) for j in range(1, M * s + 1)) * Pp / (Nt * prob.Ne) for s in range(Ntau + 1)])
    if not S["modified"]:
        U_th = U_th ** (1 / p)
    V_l = np.array([lam_old[n] * S["v"] for n in range(Ntau + 1)]) if lam_old is not None else np.zeros_like(U_T)
    V_g = rng.standard_normal((Ntau + 1, prob.Ne))
    V_g[Ntau] = 0.0
    return (U_T, U_th), (V_l, V_g)


CASES = [  # nx, ny, mx, my, Nt, Ntau, p, modified objective (Sec. 7.1) or the power mean
    (8, 6, 1, 1, 12, 3, 2.0, True),
    (8, 6, 2, 1, 12, 4, 2.0, True),
    (7, 9, 1, 2, 10, 5, 2.0, True),
    (8, 6, 1, 1, 12, 3, 8.0, True),
    (6, 6, 1, 1, 8, 2, 8.0, True),
    (8, 6, 1, 1, 12, 3, 2.0, False),
    (7, 9, 2, 1, 10, 5, 2.0, False),
    (8, 6, 1, 1, 12, 4, 8.0, False),
]


@pytest.mark.parametrize("nx,ny,mx,my,Nt,Ntau,p,modified", CASES)
def test_oneshot_pass_with_a_changed_design_matches_the_closed_form(nx, ny, mx, my, Nt, Ntau, p, modified):
    dt, rho_a, rho_b = 0.011, 0.6, 0.75
    S = _setup(nx, ny, mx, my, Nt, Ntau, p, dt, rho_a, rho_b, modified)
    cf = _closed_form(S, Nt, Ntau, p, dt)
    U_old, V_old = _old_states(S, Nt, Ntau, p, dt, cf.get("lam_old"), np.random.default_rng(3))
    out = oneshot_pass(Operator(S["prob"], np.full(nx * ny, rho_b)), U_old, V_old)
    v = S["v"]
    scale = np.max(np.abs(v))
    for j in range(Nt + 1):                                 # corrected and uncorrected rows
        assert np.max(np.abs(out["T_hist"][j] - cf["tau"][j] * v)) < 1e-12 * scale, j
    assert abs(out["Theta"] - cf["Theta"]) < 1e-11 * abs(cf["Theta"])
    # the design change is visible: the one-shot estimate is not the old design's history
    assert abs(cf["tau"][Nt] - U_old[0][Ntau] @ v / (v @ v)) > 1e-3 * abs(cf["tau"][Nt])
    if p != 2:
        return
    lam = out["V"][0]
    lam_scale = np.max(np.abs(cf["lam_new"])) * scale
    for n in range(Ntau + 1):
        assert np.max(np.abs(lam[n] - cf["lam_new"][n] * v)) < 1e-11 * lam_scale, n
    qk, qm = _element_forms(S)
    g = cf["gk"] * qk + cf["gm"] * qm
    assert np.max(np.abs(out["grad"] - g)) < 1e-10 * np.max(np.abs(g))
    assert np.max(np.abs(g)) > 0 and abs(cf["gm"]) > 1e-3 * abs(cf["gk"])   # both terms matter


def test_gradient_does_not_depend_on_the_old_g_states():
    """The old g enters F_g and G_g alike and cancels from their difference (Eq. 4.14)."""
    nx, ny, mx, my, Nt, Ntau, p, dt = 8, 6, 1, 1, 12, 3, 2.0, 0.011
    S = _setup(nx, ny, mx, my, Nt, Ntau, p, dt, 0.6, 0.75)
    cf = _closed_form(S, Nt, Ntau, p, dt)
    op = Operator(S["prob"], np.full(nx * ny, 0.75))
    grads = []
    for seed in (1, 2):
        U_old, V_old = _old_states(S, Nt, Ntau, p, dt, cf["lam_old"], np.random.default_rng(seed))
        grads.append(oneshot_pass(op, U_old, V_old)["grad"])
    assert np.max(np.abs(grads[0] - grads[1])) < 1e-12 * np.max(np.abs(grads[0]))


# ------------------------------------------------------------------ planted mistakes

def _planted(name):
    """Plausible mistakes, each planted in the oracle: G_adj reading T_{M(s+1)} instead of
    T_{Ms+1}; the coarse theta increment divided by Nt Ne instead of Ntau Ne; the fine adjoint's
    sensitivity divided by Ntau instead of Nt; a coarse step of dt; the adjoint source scale
    Theta^(-p) / Ne instead of Theta^(1-p) / Ne (Eq. 4.6); the capacity term of Eq. 4.7 dropped
    or with its sign flipped."""
    import importlib
    import sys

    importlib.import_module("oracle.parareal")
    PR = sys.modules["oracle.parareal"]
    from oracle.stepping import accumulate_theta, sensitivity_term

    ST = sys.modules["oracle.stepping"]

    def source_scale(prob, Theta):
        return prob.p / prob.Ne if prob.modified_objective else Theta ** (-prob.p) / prob.Ne

    def G_adj_row(op, s, lam, g, T_hist, Theta):
        prob = op.prob
        k, kp = prob.M * (s + 1), max(prob.M * s + 1 - prob.M, 0)
        ln = op.step_adjoint(lam, T_hist[k], Theta, prob.dtau)
        return ln, g - sensitivity_term(op, ln, T_hist[k], T_hist[kp], prob.dtau) / prob.Ntau

    def G_pri_divisor(op, s, T_, th):
        prob = op.prob
        Tn = op.step_primal(np.asarray(T_, dtype=np.float64), prob.M * (s + 1), prob.dtau)
        return Tn, accumulate_theta(prob, th, Tn, prob.Nt)

    def G_pri_step(op, s, T_, th):
        prob = op.prob
        Tn = op.step_primal(np.asarray(T_, dtype=np.float64), prob.M * (s + 1), prob.dt)
        return Tn, accumulate_theta(prob, th, Tn, prob.Ntau)

    def F_adj_divisor(op, s, lam, g, T_hist, Theta):
        prob = op.prob
        lam, g = np.array(lam, dtype=np.float64), np.array(g, dtype=np.float64)
        for j in range(prob.M * (s + 1), prob.M * s, -1):
            lam = op.step_adjoint(lam, T_hist[j], Theta, prob.dt)
            g = g - sensitivity_term(op, lam, T_hist[j], T_hist[j - 1], prob.dt) / prob.Ntau
        return lam, g

    def sens_without_capacity(op, lam, T_j, T_jm1, dt):
        return sensitivity_term(op, lam, T_j, T_jm1, dt) - op.dc * np.einsum(
            "ei,ij,ej->e", lam[op.en], op.Me, (T_j - T_jm1)[op.en] / dt)

    def sens_capacity_sign(op, lam, T_j, T_jm1, dt):
        return sensitivity_term(op, lam, T_j, T_jm1, dt) - 2.0 * op.dc * np.einsum(
            "ei,ij,ej->e", lam[op.en], op.Me, (T_j - T_jm1)[op.en] / dt)

    table = {"G_adj_row": (PR, "G_adj", G_adj_row), "G_pri_divisor": (PR, "G_pri", G_pri_divisor),
             "G_pri_step": (PR, "G_pri", G_pri_step), "F_adj_divisor": (PR, "F_adj", F_adj_divisor),
             "source_exponent": (ST, "adjoint_source_scale", source_scale),
             "sens_without_capacity": (PR, "sensitivity_term", sens_without_capacity),
             "sens_capacity_sign": (PR, "sensitivity_term", sens_capacity_sign)}
    return table[name]


@pytest.mark.parametrize("name", ["G_adj_row", "G_pri_divisor", "G_pri_step", "F_adj_divisor", "source_exponent",
                                  "sens_without_capacity", "sens_capacity_sign"])
def test_a_planted_mistake_fails_the_closed_form(monkeypatch, name):
    module, attr, fn = _planted(name)
    monkeypatch.setattr(module, attr, fn)
    failed = False
    for case in CASES:
        try:
            test_oneshot_pass_with_a_changed_design_matches_the_closed_form(*case)
        except AssertionError:
            failed = True
            break
    assert failed, name
