"""Parareal propagators, the modified forward / vanilla reverse Parareal, and the
one-shot pass (Sec. 4.2-4.4, Algorithms 1-3; PLT variant of Sec. 7).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Indexing (Sec. 4.2): tau_n = t_{M n}, M = Nt / Ntau.  Slice s (0-based) spans the fine
steps j = M s + 1 .. M (s + 1).

Primal states u_n = (T_{Mn}, theta_{Mn}) (Sec. 4.4).
  F_pri(s, u_s): M applications of H_pri (Alg. 1) with step dt and divisor Nt Ne.
  G_pri(s, u_s): one application of H_pri with dt -> dtau, Nt -> Ntau and the previous
                 time index n-1 -> n-M: it solves for T_{M(s+1)} with the load q_{M(s+1)}.
Adjoint states v_n = (lambda_{Mn+1}, g_{Mn+1}), v_Ntau = 0 (Sec. 4.4).
  F_adj(s, v_{s+1}): M applications of H_adj (Alg. 2), j = M(s+1) .. Ms+1.
  G_adj(s, v_{s+1}): one application of H_adj with dt -> dtau, Nt -> Ntau, n+1 -> n+M and
                 n-1 -> n-M: it solves for lambda_k, k = Ms+1, from lambda_{k+M}, using T_k
                 and T_{k-M}; for s = 0 the index k-M is negative and is read as T_0.

Readings where the paper is silent (all listed in the design notes):
  * G(u_n^old) in the one-shot correction is recomputed with the current design.
  * The correction acts on (T, theta) and (lambda, g) themselves, Eq. 4.9 and 4.14.
  * The adjoint source of both F_adj and G_adj uses the corrected Theta = theta_Nt of
    the same pass, and the history T of the same pass.
  * The modified forward Parareal (Sec. 4.3) returns the corrected T at the coarse points
    and the uncorrected intermediates of F(u_s^old) between them.
"""
from __future__ import annotations

import numpy as np

from .stepping import Operator, accumulate_theta, sensitivity_term, sequential_pass


# ------------------------------------------------------------------ propagators

def F_pri(op: Operator, s: int, T: np.ndarray, theta: float):
    """Fine primal propagator over slice s.  Returns (T_end, theta_end, inter) where
    inter[i] is T_{Ms+1+i}, i = 0..M-1 (the last one equals T_end)."""
    prob = op.prob
    M = prob.M
    inter = np.zeros((M, prob.Nn))
    T = np.asarray(T, dtype=np.float64).copy()
    for i in range(M):
        j = M * s + 1 + i
        T = op.step_primal(T, j, prob.dt)
        theta = accumulate_theta(prob, theta, T, prob.Nt)
        inter[i] = T
    return T, theta, inter


def G_pri(op: Operator, s: int, T: np.ndarray, theta: float):
    """Coarse primal propagator over slice s: one step of size dtau."""
    prob = op.prob
    j_end = prob.M * (s + 1)
    T_new = op.step_primal(np.asarray(T, dtype=np.float64), j_end, prob.dtau)
    theta_new = accumulate_theta(prob, theta, T_new, prob.Ntau)
    return T_new, theta_new


def F_adj(op: Operator, s: int, lam: np.ndarray, g: np.ndarray, T_hist: np.ndarray, Theta: float):
    """Fine adjoint propagator over slice s, from v_{s+1} to an estimate of v_s."""
    prob = op.prob
    M = prob.M
    lam = np.asarray(lam, dtype=np.float64).copy()
    g = np.asarray(g, dtype=np.float64).copy()
    for j in range(M * (s + 1), M * s, -1):
        lam = op.step_adjoint(lam, T_hist[j], Theta, prob.dt)
        g = g - sensitivity_term(op, lam, T_hist[j], T_hist[j - 1], prob.dt) / prob.Nt
    return lam, g


def G_adj(op: Operator, s: int, lam: np.ndarray, g: np.ndarray, T_hist: np.ndarray, Theta: float):
    """Coarse adjoint propagator over slice s: one reverse step of size dtau."""
    prob = op.prob
    M = prob.M
    k = M * s + 1
    k_prev = max(k - M, 0)
    lam_new = op.step_adjoint(np.asarray(lam, dtype=np.float64), T_hist[k], Theta, prob.dtau)
    g_new = np.asarray(g, dtype=np.float64) - sensitivity_term(op, lam_new, T_hist[k], T_hist[k_prev], prob.dtau) / prob.Ntau
    return lam_new, g_new


# ------------------------------------------------------------------ coarse states

def coarse_states_from_sequential(op: Operator, seq: dict | None = None):
    """Coarse states of the sequential solution: U = (T_{Mn}, theta_{Mn}), n = 0..Ntau,
    and V = (lambda_{Mn+1}, g_{Mn+1}), n = 0..Ntau (V_Ntau = 0).  These are the warm start
    produced by the sequential first iteration of Alg. 3."""
    prob = op.prob
    if seq is None:
        seq = sequential_pass(op)
    M, Ntau = prob.M, prob.Ntau
    idx = np.arange(Ntau + 1) * M
    U_T = seq["T_hist"][idx].copy()
    U_th = seq["theta"][idx].copy()
    V_lam = seq["lam"][idx + 1].copy()
    V_g = seq["g"][idx + 1].copy()
    return (U_T, U_th), (V_lam, V_g), seq


# ------------------------------------------------------------------ Parareal iterations

def _coarse_fns(op: Operator, coarse):
    """The coarse propagators: the fine-mesh G of Sec. 4.4, or those of a coarse-mesh object
    (``oracle.coarse_mesh.CoarseMesh``, Sec. 7.3 future work)."""
    if coarse is None:
        return (lambda s, T, th: G_pri(op, s, T, th)), (lambda s, l, g, Th, Tt: G_adj(op, s, l, g, Th, Tt))
    return coarse.G_pri, coarse.G_adj


def primal_iteration(op: Operator, U_old, plt: bool = False, coarse=None):
    """One modified forward Parareal iteration (Eq. 4.9 with the history of Sec. 4.3)
    from the guess U_old = (T[Ntau+1, Nn], theta[Ntau+1]).  With plt=True the coarse
    propagator is identically zero (Eq. 7.1-7.2); ``coarse`` replaces G (coarse mesh)."""
    Gp, _ = _coarse_fns(op, coarse)
    prob = op.prob
    M, Ntau = prob.M, prob.Ntau
    U_T_old, U_th_old = U_old
    F_T = np.zeros((Ntau, prob.Nn)); F_th = np.zeros(Ntau)
    G_T = np.zeros((Ntau, prob.Nn)); G_th = np.zeros(Ntau)
    T_hist = np.zeros((prob.Nt + 1, prob.Nn))
    for s in range(Ntau):                                  # parallel part
        F_T[s], F_th[s], inter = F_pri(op, s, U_T_old[s], U_th_old[s])
        T_hist[M * s + 1: M * (s + 1) + 1] = inter
        if not plt:
            G_T[s], G_th[s] = Gp(s, U_T_old[s], U_th_old[s])
    U_T = np.zeros_like(U_T_old); U_th = np.zeros_like(U_th_old)
    U_T[0], U_th[0] = U_T_old[0], U_th_old[0]             # u_0^k = u_0
    T_hist[0] = U_T[0]
    for s in range(Ntau):                                  # sequential correction
        if plt:
            gT, gth = np.zeros(prob.Nn), 0.0
        else:
            gT, gth = Gp(s, U_T[s], U_th[s])
        U_T[s + 1] = gT + F_T[s] - G_T[s]
        U_th[s + 1] = gth + F_th[s] - G_th[s]
        T_hist[M * (s + 1)] = U_T[s + 1]
    return dict(U=(U_T, U_th), T_hist=T_hist, Theta=float(U_th[Ntau]),
                F=(F_T, F_th), G_old=(G_T, G_th))


def adjoint_iteration(op: Operator, V_old, T_hist: np.ndarray, Theta: float, plt: bool = False, coarse=None):
    """One reverse vanilla Parareal iteration (Eq. 4.10) from the guess V_old =
    (lam[Ntau+1, Nn], g[Ntau+1, Ne]); v_Ntau = 0 always."""
    _, Ga = _coarse_fns(op, coarse)
    prob = op.prob
    Ntau = prob.Ntau
    V_lam_old, V_g_old = V_old
    F_l = np.zeros((Ntau, prob.Nn)); F_g = np.zeros((Ntau, prob.Ne))
    G_l = np.zeros((Ntau, prob.Nn)); G_g = np.zeros((Ntau, prob.Ne))
    for s in range(Ntau):                                  # parallel part
        F_l[s], F_g[s] = F_adj(op, s, V_lam_old[s + 1], V_g_old[s + 1], T_hist, Theta)
        if not plt:
            G_l[s], G_g[s] = Ga(s, V_lam_old[s + 1], V_g_old[s + 1], T_hist, Theta)
    V_lam = np.zeros_like(V_lam_old); V_g = np.zeros_like(V_g_old)
    for s in range(Ntau - 1, -1, -1):                      # sequential correction, reversed
        if plt:
            gl, gg = np.zeros(prob.Nn), np.zeros(prob.Ne)
        else:
            gl, gg = Ga(s, V_lam[s + 1], V_g[s + 1], T_hist, Theta)
        V_lam[s] = gl + F_l[s] - G_l[s]
        V_g[s] = gg + F_g[s] - G_g[s]
    return dict(V=(V_lam, V_g), grad=V_g[0].copy(), F=(F_l, F_g), G_old=(G_l, G_g))


def oneshot_pass(op: Operator, U_old, V_old, plt: bool = False, coarse=None) -> dict:
    """The iteration body of Alg. 3: one modified forward Parareal iteration and one reverse
    vanilla Parareal iteration, each warm-started from the previous design iteration's
    coarse states; Theta = theta_Nt and grad = g_1 (Sec. 4.4, four-step procedure).
    ``coarse``: coarse propagators on a coarsened mesh (``oracle.coarse_mesh.CoarseMesh``)."""
    pri = primal_iteration(op, U_old, plt=plt, coarse=coarse)
    adj = adjoint_iteration(op, V_old, pri["T_hist"], pri["Theta"], plt=plt, coarse=coarse)
    out = dict(pri)
    out.update(V=adj["V"], grad=adj["grad"], F_adj=adj["F"], G_adj_old=adj["G_old"])
    out["F_pri"] = pri["F"]
    out["G_pri_old"] = pri["G_old"]
    return out


def initial_guess_primal(op: Operator, coarse=None):
    """u_{n+1}^0 = G_pri(u_n^0) from u_0 (Sec. 5.2)."""
    Gp, _ = _coarse_fns(op, coarse)
    prob = op.prob
    U_T = np.zeros((prob.Ntau + 1, prob.Nn)); U_th = np.zeros(prob.Ntau + 1)
    if prob.T0 is not None:
        U_T[0] = prob.T0
    for s in range(prob.Ntau):
        U_T[s + 1], U_th[s + 1] = Gp(s, U_T[s], U_th[s])
    return U_T, U_th


def initial_guess_adjoint(op: Operator, T_hist: np.ndarray, Theta: float, coarse=None):
    """v_{n-1}^0 = G_adj(v_n^0) from v_Ntau = 0 (Sec. 5.2)."""
    _, Ga = _coarse_fns(op, coarse)
    prob = op.prob
    V_lam = np.zeros((prob.Ntau + 1, prob.Nn)); V_g = np.zeros((prob.Ntau + 1, prob.Ne))
    for s in range(prob.Ntau - 1, -1, -1):
        V_lam[s], V_g[s] = Ga(s, V_lam[s + 1], V_g[s + 1], T_hist, Theta)
    return V_lam, V_g


def parareal(op: Operator, k: int, plt: bool = False, coarse=None) -> dict:
    """k-iteration Parareal of the preliminary tests (Sec. 5.2): coarse initial guess,
    k modified forward iterations, then a coarse adjoint initial guess from the final
    history and k reverse iterations."""
    U = initial_guess_primal(op, coarse=coarse)
    pri = None
    for _ in range(k):
        pri = primal_iteration(op, U, plt=plt, coarse=coarse)
        U = pri["U"]
    if pri is None:
        raise ValueError("k must be >= 1")
    V = initial_guess_adjoint(op, pri["T_hist"], pri["Theta"], coarse=coarse)
    adj = None
    for _ in range(k):
        adj = adjoint_iteration(op, V, pri["T_hist"], pri["Theta"], plt=plt, coarse=coarse)
        V = adj["V"]
    return dict(U=U, T_hist=pri["T_hist"], Theta=pri["Theta"], V=V, grad=adj["grad"])
