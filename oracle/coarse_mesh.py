"""Coarse propagators on a coarsened spatial mesh: the remedy for the sequential coarse sweep
that the paper proposes as future work (Sec. 7.3).  G_pri and G_adj take their single step of
size dtau on the mesh of spacing 2h instead of h; F and the corrections stay on the fine mesh.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper names the idea but not its construction, so every piece below is a reading:

* Coarse mesh: nx/2 x ny/2 square elements of side 2h (nx and ny even).  Coarse node (I, J)
  sits on fine node (2I, 2J).  A coarse node is a sink (Dirichlet) node when its fine node is.
* Coarse design: the density of a coarse element is the mean of its four fine elements; the
  same SIMP laws give k and c, and the element source density is the mean of the four fine
  ones.  The coarse operators are the finite-element operators of that design on the 2h mesh
  (assembled exactly as on the fine mesh).
* Transfers: R takes a fine nodal state to the coarse mesh by injection (the values at the
  coarse nodes); P takes a coarse nodal state to the fine mesh by bilinear interpolation
  (weights 1, 1/2, 1/4), zero at fine sink nodes.  R P is the identity on the coarse free
  nodes.  A nodal source that is a derivative of a sum over fine nodes (the adjoint source
  T^(p-1)) is restricted by P^T, as a load vector is: for a uniform fine load P^T f_h equals
  the load vector assembled on the coarse mesh.
* G_pri(u) = (P x, theta increment of P x) with x the coarse backward-Euler step of size dtau
  from R T: (C_H/dtau + K_H) x = C_H/dtau R T + q_H(t_{M(s+1)}).  theta is updated from the
  fine-mesh p-norm of P x with the divisor Ntau Ne, exactly as the fine-mesh G does.
* G_adj(v) = (P z, g increment of P z) with (C_H/dtau + K_H) z = C_H/dtau R lam + P^T (scale
  T_k^(p-1)), scale = Theta^(1-p)/Ne (or p/Ne for the modified objective), and the g increment
  the fine-mesh sensitivity term of P z with T_k and T_{k-M} (Eq. 4.7), as in the fine-mesh G.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fem import Problem
from .stepping import Operator, accumulate_theta, adjoint_source_scale, sensitivity_term


def coarse_problem(prob: Problem) -> Problem:
    """The problem on the 2h mesh: same materials, objective and time data, coarse sink nodes."""
    if prob.nx % 2 or prob.ny % 2:
        raise ValueError("the coarse mesh needs an even number of elements per direction")
    nxH, nyH = prob.nx // 2, prob.ny // 2
    dfine = np.asarray(prob.dirichlet, dtype=np.uint8).reshape(prob.ny + 1, prob.nx + 1)
    dH = dfine[::2, ::2].reshape(-1).copy()
    q = None
    if prob.q_elem is not None:
        q = coarse_elements(np.asarray(prob.q_elem, dtype=np.float64), prob.nx, prob.ny)
    return Problem(nx=nxH, ny=nyH, h=2.0 * prob.h, material=prob.material, Nt=prob.Nt, dt=prob.dt,
                   Ntau=prob.Ntau, p=prob.p, dirichlet=dH, q_elem=q, q_time=prob.q_time, T0=None,
                   modified_objective=prob.modified_objective)


def coarse_elements(v: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Mean of the four fine elements of every coarse element (row-major element order)."""
    a = np.asarray(v, dtype=np.float64).reshape(ny, nx)
    return (0.25 * (a[0::2, 0::2] + a[0::2, 1::2] + a[1::2, 0::2] + a[1::2, 1::2])).reshape(-1)


def prolongation(prob: Problem) -> sp.csr_matrix:
    """P: coarse nodal values -> fine nodal values, bilinear interpolation, zero rows at fine
    sink nodes and zero columns at coarse sink nodes."""
    nx, ny = prob.nx, prob.ny
    nxH, nyH = nx // 2, ny // 2
    rows, cols, vals = [], [], []
    for iy in range(ny + 1):
        for ix in range(nx + 1):
            i = iy * (nx + 1) + ix
            ys = [(iy // 2, 1.0)] if iy % 2 == 0 else [(iy // 2, 0.5), (iy // 2 + 1, 0.5)]
            xs = [(ix // 2, 1.0)] if ix % 2 == 0 else [(ix // 2, 0.5), (ix // 2 + 1, 0.5)]
            for J, wy in ys:
                for I, wx in xs:
                    rows.append(i)
                    cols.append(J * (nxH + 1) + I)
                    vals.append(wx * wy)
    P = sp.csr_matrix((vals, (rows, cols)), shape=((nx + 1) * (ny + 1), (nxH + 1) * (nyH + 1)))
    dF = np.asarray(prob.dirichlet).reshape(-1) != 0
    dH = np.asarray(coarse_problem(prob).dirichlet).reshape(-1) != 0
    return (sp.diags((~dF).astype(float)) @ P @ sp.diags((~dH).astype(float))).tocsr()


def injection(prob: Problem, T: np.ndarray) -> np.ndarray:
    """R: the fine nodal values at the coarse nodes (zero at coarse sink nodes)."""
    a = np.asarray(T, dtype=np.float64).reshape(prob.ny + 1, prob.nx + 1)[::2, ::2].reshape(-1).copy()
    dH = np.asarray(coarse_problem(prob).dirichlet).reshape(-1) != 0
    a[dH] = 0.0
    return a


class CoarseMesh:
    """The coarse-mesh propagators of one design rho (fine-mesh operator ``op``)."""

    def __init__(self, op: Operator):
        self.op = op
        self.prob = op.prob
        self.probH = coarse_problem(op.prob)
        self.opH = Operator(self.probH, coarse_elements(op.rho, op.prob.nx, op.prob.ny))
        self.P = prolongation(op.prob)

    def R(self, T: np.ndarray) -> np.ndarray:
        return injection(self.prob, T)

    def G_pri(self, s: int, T: np.ndarray, theta: float):
        prob, opH = self.prob, self.opH
        j_end = prob.M * (s + 1)
        x = opH.solve(prob.dtau, opH.C @ self.R(T) / prob.dtau + opH.load(j_end))
        T_new = self.P @ x
        return T_new, accumulate_theta(prob, theta, T_new, prob.Ntau)

    def G_adj(self, s: int, lam: np.ndarray, g: np.ndarray, T_hist: np.ndarray, Theta: float):
        prob, opH = self.prob, self.opH
        k = prob.M * s + 1
        k_prev = max(k - prob.M, 0)
        src = adjoint_source_scale(prob, Theta) * T_hist[k] ** (prob.p - 1.0)
        z = opH.solve(prob.dtau, opH.C @ self.R(lam) / prob.dtau + self.P.T @ src)
        lam_new = self.P @ z
        g_new = np.asarray(g, dtype=np.float64) - sensitivity_term(self.op, lam_new, T_hist[k], T_hist[k_prev],
                                                                   prob.dtau) / prob.Ntau
        return lam_new, g_new
