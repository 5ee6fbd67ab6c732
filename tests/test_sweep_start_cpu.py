"""The start of a correction-sweep step (ptg_solve.initial_guess), pinned on the oracle's
one-shot pass (Sec. 4.3-4.4): the answer of step s is G(u_s^new) = u_{s+1}^new - F[s] + G_old[s]
(Eq. 4.9), and the start is G_old[s] plus the polynomial extrapolation of the increments
d_i = u_{s-i}^new - F[s-1-i] of the previous steps (order n - 1).  The starts of higher order
must land closer to the answer, primal and adjoint (Eq. 4.14, mirrored in time): that is what
lets the default (n = 4) cut the sweep's CG iterations.  The formulas are written here as the
kernels state them; the oracle supplies every state."""
from __future__ import annotations

import numpy as np

import workloads as W
from oracle import Operator, coarse_states_from_sequential, oneshot_pass
from tests.problems import make_problem


def _extrapolate(G, d, m):
    if m == 1:
        return G + d[0]
    if m == 2:
        return G + 2.0 * d[0] - d[1]
    return G + 3.0 * (d[0] - d[1]) + d[2]


def _geo(v):
    return float(np.exp(np.mean(np.log(np.maximum(v, 1e-300)))))


def _start_errors(q_time, material="table1", n=24, Nt=96, Ntau=24):
    prob = make_problem(n, Nt=Nt, Ntau=Ntau, dt=1.0 / Nt, material=material, sink="left_wide", q_time=q_time)
    rho = W.rho_uniform(n, n, 7, 0.1, 0.9)
    rho_old = W.rho_warm_perturb(rho, seed=8, amp=0.02)
    U_old, V_old, _ = coarse_states_from_sequential(Operator(prob, rho_old))
    out = oneshot_pass(Operator(prob, rho), U_old, V_old)
    free = np.asarray(prob.dirichlet).reshape(-1) == 0
    # primal: the answer of step s is X[s] = G(u_s^new); increments d_i = U[s-i] - F[s-1-i]
    U, F, G = out["U"][0], out["F_pri"][0], out["G_pri_old"][0]
    X = U[1:] - F + G
    pri = {m: [] for m in (1, 2, 3)}
    for s in range(3, Ntau):
        d = [U[s - i] - F[s - 1 - i] for i in range(3)]
        for m in (1, 2, 3):
            e = _extrapolate(G[s], d, m) - X[s]
            pri[m].append(np.linalg.norm(e[free]) / np.linalg.norm(X[s][free]))
    # adjoint: the answer is Y[s] = G(v_{s+1}^new); increments d_i = V[s+1+i] - F[s+1+i]
    V, Fa, Ga = out["V"][0], out["F_adj"][0], out["G_adj_old"][0]
    Y = V[:Ntau] - Fa + Ga
    adj = {m: [] for m in (1, 2, 3)}
    for s in range(Ntau - 4, -1, -1):
        d = [V[s + 1 + i] - Fa[s + 1 + i] for i in range(3)]
        for m in (1, 2, 3):
            e = _extrapolate(Ga[s], d, m) - Y[s]
            adj[m].append(np.linalg.norm(e[free]) / np.linalg.norm(Y[s][free]))
    return ({m: _geo(v) for m, v in pri.items()}, {m: _geo(v) for m, v in adj.items()})


def test_higher_order_sweep_starts_land_closer_with_a_smooth_source():
    # the uniform source of the benchmark configurations: the increments are smooth in time
    for material in ("simp_k", "table1"):
        for g in _start_errors(None, material):
            assert g[3] < g[2] < g[1], g
            assert g[3] < 0.2 * g[1], g


def test_sweep_starts_with_an_oscillating_source():
    # the paper's q(t) = (1 - t)(1 + cos 50 t)/2 turns by about 2 rad per coarse step here: the
    # linear extrapolation still helps, the quadratic one gains little over the previous
    # increment alone, and none is worse than that by more than a small factor
    pri, adj = _start_errors(W.q_time_paper(96, 1.0 / 96))
    for g in (pri, adj):
        assert g[2] < g[1], g
        assert g[3] < 1.5 * g[1], g
