"""Dense all-at-once space-time solves for tiny grids (Eq. 2.8-2.9, 4.3-4.5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The whole history S = (T_1 .. T_Nt) solves the block lower-bidiagonal system M S = Q
(Eq. 2.8-2.9) with (C/dt + K) on the diagonal and -C/dt below it.  The adjoint
Lambda solves M^T Lambda = Nt (dTheta/dS)^T (Eq. 4.3) and the gradient is
-(1/Nt) Lambda^T dR/drho (Eq. 4.5), with dR/drho assembled column by column from
single-element matrices.  Everything is dense and restricted to the free nodes, so
this is only for grids of a few dozen nodes.
"""
from __future__ import annotations

import numpy as np

from .fem import Problem, element_matrices, element_nodes, simp
from .stepping import Operator


def _dense(op: Operator):
    f = op.fidx
    K = op.K.toarray()[np.ix_(f, f)]
    C = op.C.toarray()[np.ix_(f, f)]
    return K, C


def solve_all_at_once(op: Operator):
    """Solve M S = Q densely.  Returns T_hist[Nt+1, Nn] (row 0 = T_0)."""
    prob = op.prob
    Nt, dt = prob.Nt, prob.dt
    K, C = _dense(op)
    nf = K.shape[0]
    Mbig = np.zeros((Nt * nf, Nt * nf))
    Q = np.zeros(Nt * nf)
    T0 = np.zeros(prob.Nn) if prob.T0 is None else np.asarray(prob.T0, dtype=np.float64)
    for j in range(Nt):
        Mbig[j * nf:(j + 1) * nf, j * nf:(j + 1) * nf] = C / dt + K
        if j > 0:
            Mbig[j * nf:(j + 1) * nf, (j - 1) * nf:j * nf] = -C / dt
        Q[j * nf:(j + 1) * nf] = op.load(j + 1)[op.fidx]
    Q[:nf] += (C / dt) @ T0[op.fidx]
    S = np.linalg.solve(Mbig, Q)
    T_hist = np.zeros((Nt + 1, prob.Nn))
    T_hist[0] = T0
    for j in range(Nt):
        T_hist[j + 1, op.fidx] = S[j * nf:(j + 1) * nf]
    return T_hist, Mbig


def adjoint_all_at_once(op: Operator, T_hist: np.ndarray, Mbig: np.ndarray):
    """Solve M^T Lambda = Nt (dTheta/dS)^T densely and form the gradient of Eq. 4.5.

    dTheta/dS is differentiated directly from Theta = (Nt Ne)^(-1/p) ||S||_p (Eq. 2.12):
    dTheta/dS_i = (Nt Ne)^(-1/p) ||S||_p^(1-p) S_i^(p-1).
    dR/drho_e is assembled per element e from its element matrices: block j holds
    dc_e Me (T_j - T_{j-1})/dt + dk_e Ke T_j restricted to the element's free nodes.
    """
    prob = op.prob
    Nt, Ne, p, dt = prob.Nt, prob.Ne, prob.p, prob.dt
    nf = len(op.fidx)
    S = np.concatenate([T_hist[j, op.fidx] for j in range(1, Nt + 1)])
    normS = np.sum(S ** p) ** (1.0 / p)
    dTheta_dS = (Nt * Ne) ** (-1.0 / p) * normS ** (1.0 - p) * S ** (p - 1.0)
    Lam = np.linalg.solve(Mbig.T, Nt * dTheta_dS)
    _, _, dk, dc = simp(op.rho, prob.material)
    Ke, Me, _ = element_matrices(prob.h)
    en = element_nodes(prob.nx, prob.ny)
    pos = -np.ones(prob.Nn, dtype=int)
    pos[op.fidx] = np.arange(nf)
    dR = np.zeros((Nt * nf, Ne))
    for e in range(Ne):
        nodes = en[e]
        for j in range(1, Nt + 1):
            col = dc[e] * Me @ (T_hist[j, nodes] - T_hist[j - 1, nodes]) / dt + dk[e] * Ke @ T_hist[j, nodes]
            for a in range(4):
                if pos[nodes[a]] >= 0:
                    dR[(j - 1) * nf + pos[nodes[a]], e] += col[a]
    grad = -(1.0 / Nt) * Lam @ dR
    lam = np.zeros((Nt + 2, prob.Nn))
    for j in range(Nt):
        lam[j + 1, op.fidx] = Lam[j * nf:(j + 1) * nf]
    Theta = (Nt * Ne) ** (-1.0 / p) * normS
    return lam, grad, Theta
