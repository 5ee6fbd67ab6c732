"""Sequential backward Euler, objective and discrete adjoint (Sec. 2.2, 4.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Primal (Eq. 2.7):   C (T_j - T_{j-1}) / dt + K T_j = q_j,  j = 1..Nt,  T_0 given.
Objective (Eq. 2.11): Theta = ( sum_j ||T_j||_p^p / (Nt Ne) )^(1/p); the p-norm runs
                    over every node (Dirichlet nodes contribute 0) and the divisor
                    is the element count, exactly as printed.  The cumulative objective
                    theta_j = (theta_{j-1}^p + ||T_j||_p^p / (Nt Ne))^(1/p) (Sec. 4.4).
                    Modified objective (Sec. 7.1): Theta~ = Theta^p = sum_j ||T_j||_p^p / (Nt Ne),
                    cumulative theta~_j = theta~_{j-1} + ||T_j||_p^p / (Nt Ne).
Adjoint (Eq. 4.4-4.6): lambda_{Nt+1} = 0,
                    C (lambda_j - lambda_{j+1}) / dt + K lambda_j = Theta^(1-p)/Ne T_j^(p-1);
                    for Theta~ the source is p/Ne T_j^(p-1) (Sec. 7.1).
Gradient (Eq. 4.7): dTheta/drho = -(1/Nt) sum_j lambda_j^T (dC/drho (T_j - T_{j-1})/dt + dK/drho T_j).

Linear solves: the free-node block of (C/dt + K) is factored once per step size and reused:
by banded Cholesky (LAPACK via scipy.linalg.cholesky_banded) while the half-bandwidth (nx + 1
in the node numbering) is at most BAND_MAX, and by a sparse direct LU (SuperLU via
scipy.sparse.linalg.splu, minimum-degree ordering) on wider grids, where the banded factor
costs minutes (512 x 512: 272 s against 2 s).  Both solve the same system exactly up to
rounding; a pin checks that they agree.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .fem import Problem, assemble, element_matrices, element_nodes, simp


BAND_MAX = 300   # widest half-bandwidth factored as a band (wider: sparse LU)


class Operator:
    """The discrete operators of one design rho (Sec. 2.2).  solver: "auto" (band Cholesky up to
    BAND_MAX, sparse LU beyond), "band" or "lu"."""

    def __init__(self, prob: Problem, rho: np.ndarray, solver: str = "auto"):
        self.solver = solver
        self.prob = prob
        self.rho = np.asarray(rho, dtype=np.float64).copy()
        self.K, self.C, self.f = assemble(prob, self.rho)
        self.k, self.c, self.dk, self.dc = simp(self.rho, prob.material)
        self.free = np.asarray(prob.dirichlet).reshape(-1) == 0
        self.fidx = np.nonzero(self.free)[0]
        self.Ke, self.Me, _ = element_matrices(prob.h)
        self.en = element_nodes(prob.nx, prob.ny)
        self.q_time = (np.ones(prob.Nt + 1) if prob.q_time is None
                       else np.asarray(prob.q_time, dtype=np.float64))
        self._factors: dict[float, tuple[np.ndarray, int]] = {}

    # -- linear algebra ------------------------------------------------------
    def _factor(self, dt: float):
        key = float(dt)
        if key not in self._factors:
            A = (self.C / dt + self.K).tocsr()[self.fidx][:, self.fidx].tocoo()
            u = int(np.max(A.col - A.row)) if A.nnz else 0
            if self.solver == "lu" or (self.solver == "auto" and u > BAND_MAX):
                self._factors[key] = ("lu", spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A"))
            else:
                n = A.shape[0]
                ab = np.zeros((u + 1, n))
                upper = A.col >= A.row
                ab[u + A.row[upper] - A.col[upper], A.col[upper]] = A.data[upper]
                self._factors[key] = ("band", sla.cholesky_banded(ab, lower=False))
        return self._factors[key]

    def solve(self, dt: float, rhs: np.ndarray) -> np.ndarray:
        """Solve (C/dt + K) x = rhs on the free nodes; x = 0 on Dirichlet nodes."""
        kind, f = self._factor(dt)
        x = np.zeros(self.prob.Nn)
        if kind == "lu":
            x[self.fidx] = f.solve(np.ascontiguousarray(rhs[self.fidx]))
        else:
            x[self.fidx] = sla.cho_solve_banded((f, False), rhs[self.fidx])
        return x

    def load(self, j: int) -> np.ndarray:
        """q_j, the load vector at t_j."""
        return self.q_time[j] * self.f

    def step_primal(self, T_prev: np.ndarray, j: int, dt: float) -> np.ndarray:
        """One backward-Euler solve ending at t_j from T_prev (Alg. 1, first line)."""
        return self.solve(dt, self.C @ T_prev / dt + self.load(j))

    def step_adjoint(self, lam_next: np.ndarray, T_j: np.ndarray, Theta: float, dt: float) -> np.ndarray:
        """One reverse adjoint solve (Alg. 2, first line)."""
        src = adjoint_source_scale(self.prob, Theta) * T_j ** (self.prob.p - 1.0)
        return self.solve(dt, self.C @ lam_next / dt + src)


def accumulate_theta(prob: Problem, theta_prev: float, T: np.ndarray, N: int) -> float:
    """One update of the cumulative objective with the divisor N Ne (N = Nt for H and F,
    N_tau for G): the power mean of Sec. 4.4, or the plain sum of Sec. 7.1 for Theta~."""
    inc = pnorm_p(T, prob.p) / (N * prob.Ne)
    if prob.modified_objective:
        return theta_prev + inc
    return (theta_prev ** prob.p + inc) ** (1.0 / prob.p)


def adjoint_source_scale(prob: Problem, Theta: float) -> float:
    """Factor of T_j^(p-1) in the adjoint source: Theta^(1-p)/Ne (Eq. 4.6) or p/Ne (Sec. 7.1)."""
    if prob.modified_objective:
        return prob.p / prob.Ne
    return Theta ** (1.0 - prob.p) / prob.Ne


def objective_from_modified(Theta_mod: float, grad_mod: np.ndarray, p: float):
    """Sec. 7.1: Theta = Theta~^(1/p) and grad Theta = Theta^(1-p)/p grad Theta~."""
    Theta = Theta_mod ** (1.0 / p)
    return Theta, Theta ** (1.0 - p) / p * np.asarray(grad_mod, dtype=np.float64)


def pnorm_p(T: np.ndarray, p: float) -> float:
    """||T||_p^p over all nodes (p even, Eq. 2.11)."""
    return float(np.sum(T ** p))


def objective(T_hist: np.ndarray, prob: Problem) -> float:
    """Eq. 2.11 (or Theta~ of Sec. 7.1) on a history T_hist[0..Nt]; T_0 is not part of the sum."""
    s = sum(pnorm_p(T_hist[j], prob.p) for j in range(1, prob.Nt + 1)) / (prob.Nt * prob.Ne)
    return s if prob.modified_objective else s ** (1.0 / prob.p)


def sensitivity_term(op: Operator, lam: np.ndarray, T_j: np.ndarray, T_jm1: np.ndarray, dt: float) -> np.ndarray:
    """Per element e: lambda_e^T ( dc_e Me (T_j - T_{j-1})_e / dt + dk_e Ke T_j,e ).

    This is the element-wise bracket of Eq. 4.7 (without the -1/Nt factor);
    the vectors are gathered at the element's four nodes.
    """
    lam_e = lam[op.en]                       # [Ne, 4]
    Tj_e = T_j[op.en]
    dT_e = (T_j - T_jm1)[op.en] / dt
    kterm = np.einsum("ei,ij,ej->e", lam_e, op.Ke, Tj_e)
    cterm = np.einsum("ei,ij,ej->e", lam_e, op.Me, dT_e)
    return op.dc * cterm + op.dk * kterm


def sequential_primal(op: Operator):
    """Alg. 1 applied Nt times from T_0: returns (T_hist[Nt+1, Nn], theta[Nt+1])."""
    prob = op.prob
    Nt = prob.Nt
    T = np.zeros(prob.Nn) if prob.T0 is None else np.asarray(prob.T0, dtype=np.float64).copy()
    T_hist = np.zeros((Nt + 1, prob.Nn))
    theta = np.zeros(Nt + 1)
    T_hist[0] = T
    for j in range(1, Nt + 1):
        T = op.step_primal(T, j, prob.dt)
        theta[j] = accumulate_theta(prob, theta[j - 1], T, Nt)
        T_hist[j] = T
    return T_hist, theta


def sequential_adjoint(op: Operator, T_hist: np.ndarray, Theta: float):
    """Alg. 2 applied Nt times backwards from lambda_{Nt+1} = 0, g_{Nt+1} = 0.

    Returns (lam[Nt+2, Nn], g[Nt+2, Ne]); rows 1..Nt hold lambda_j and the cumulative
    sensitivities g_j; row Nt+1 is the terminal zero; row 0 is unused (zero).
    """
    prob = op.prob
    Nt = prob.Nt
    lam = np.zeros((Nt + 2, prob.Nn))
    g = np.zeros((Nt + 2, prob.Ne))
    for j in range(Nt, 0, -1):
        lam[j] = op.step_adjoint(lam[j + 1], T_hist[j], Theta, prob.dt)
        g[j] = g[j + 1] - sensitivity_term(op, lam[j], T_hist[j], T_hist[j - 1], prob.dt) / Nt
    return lam, g


def sequential_pass(op: Operator) -> dict:
    """Sequential reference (the initialisation of Alg. 3): state, objective, adjoint, gradient."""
    T_hist, theta = sequential_primal(op)
    Theta = theta[-1]
    lam, g = sequential_adjoint(op, T_hist, Theta)
    return dict(T_hist=T_hist, theta=theta, Theta=Theta, lam=lam, g=g, grad=g[1].copy())
