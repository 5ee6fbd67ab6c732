"""Finite-element discretisation of the transient heat problem (Sec. 2.1-2.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* SIMP interpolation of capacity and conductivity, Eq. 2.5-2.6.
* Galerkin bilinear quadrilateral elements with element-wise constant k, c and q
  (Sec. 2.2).  The element matrices are integrated from the shape functions with
  2x2 Gauss quadrature, which is exact for these polynomial integrands, rather
  than typed in.
* Depth 1 (the paper non-dimensionalises with the domain depth equal to L = 1).
* Dirichlet nodes are removed from the unknowns (symmetric elimination); the
  prescribed value there is 0 (Eq. 2.1c).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Material:
    """SIMP parameters: c = cmin + (c0 - cmin) rho^pc, k = kmin + (k0 - kmin) rho^pk (Eq. 2.5-2.6)."""
    k0: float
    kmin: float
    pk: float
    c0: float
    cmin: float
    pc: float


@dataclass
class Problem:
    """Statement of one transient problem (Sec. 2 and 3).

    nx, ny   elements per side (square elements of side h)
    Nt, dt   number of backward-Euler steps and step size (t_j = j*dt)
    Ntau     number of Parareal slices (coarse steps); must divide Nt
    p        power-mean exponent (even, Eq. 2.11)
    dirichlet  uint8/bool mask over the (nx+1)(ny+1) nodes; T = lambda = 0 there
    q_elem   element-wise source density q_e (length Ne); the load at t_j is
             q_time[j] * (sum over elements of q_e * int N_i)
    q_time   time factor of the source at t_0..t_Nt
    T0       initial temperature (length Nn), zero by default (Eq. 2.1b)
    modified_objective  False: the power mean Theta of Eq. 2.11.  True: the modified
             objective Theta~ = Theta^p of Sec. 7.1, a plain sum over the steps, whose
             adjoint source is p/Ne T^(p-1) (the form the PLT comparison uses)
    """
    nx: int
    ny: int
    h: float
    material: Material
    Nt: int
    dt: float
    Ntau: int
    p: float
    dirichlet: np.ndarray
    q_elem: np.ndarray | None = None
    q_time: np.ndarray | None = None
    T0: np.ndarray | None = None
    modified_objective: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def Ne(self) -> int:
        return self.nx * self.ny

    @property
    def Nn(self) -> int:
        return (self.nx + 1) * (self.ny + 1)

    @property
    def M(self) -> int:
        if self.Nt % self.Ntau:
            raise ValueError("N_tau must divide N_t (Sec. 4.2)")
        return self.Nt // self.Ntau

    @property
    def dtau(self) -> float:
        return self.M * self.dt


# ---------------------------------------------------------------- element level

def _shape(xi: float, eta: float) -> tuple[np.ndarray, np.ndarray]:
    """Bilinear shape functions on the unit reference square and their gradients.

    Local node order is counter-clockwise from the lower-left corner:
    0 = (0,0), 1 = (1,0), 2 = (1,1), 3 = (0,1).
    """
    N = np.array([(1 - xi) * (1 - eta), xi * (1 - eta), xi * eta, (1 - xi) * eta])
    dN = np.array([[-(1 - eta), -(1 - xi)],
                   [(1 - eta), -xi],
                   [eta, xi],
                   [-eta, (1 - xi)]])
    return N, dN


def element_matrices(h: float) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Unit-coefficient element matrices of a square element of side h.

    Returns (Ke, Me, fe): Ke_ij = int grad N_i . grad N_j, Me_ij = int N_i N_j,
    fe_i = int N_i, each over the element, by 2x2 Gauss quadrature.
    """
    g = 0.5 / np.sqrt(3.0)
    pts = [0.5 - g, 0.5 + g]
    Ke = np.zeros((4, 4))
    Me = np.zeros((4, 4))
    fe = np.zeros(4)
    for xi in pts:
        for eta in pts:
            N, dN = _shape(xi, eta)
            grad = dN / h                    # d/dx = (1/h) d/dxi
            w = 0.25 * h * h                 # Gauss weight (1/4 each) times the Jacobian h^2
            Ke += w * grad @ grad.T
            Me += w * np.outer(N, N)
            fe += w * N
    return Ke, Me, fe


def element_nodes(nx: int, ny: int) -> np.ndarray:
    """Global node numbers of every element, local order SW, SE, NE, NW.  Shape [Ne, 4]."""
    ey, ex = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    sw = ey * (nx + 1) + ex
    en = np.stack([sw, sw + 1, sw + nx + 2, sw + nx + 1], axis=-1)
    return en.reshape(-1, 4)


def simp(rho: np.ndarray, mat: Material) -> tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """Eq. 2.5-2.6 and their derivatives: returns (k, c, dk/drho, dc/drho) per element."""
    rho = np.asarray(rho, dtype=np.float64)
    k = mat.kmin + (mat.k0 - mat.kmin) * rho ** mat.pk
    c = mat.cmin + (mat.c0 - mat.cmin) * rho ** mat.pc
    dk = mat.pk * (mat.k0 - mat.kmin) * rho ** (mat.pk - 1.0)
    dc = mat.pc * (mat.c0 - mat.cmin) * rho ** (mat.pc - 1.0)
    if mat.c0 == mat.cmin:
        dc = np.zeros_like(rho)
    if mat.k0 == mat.kmin:
        dk = np.zeros_like(rho)
    return k, c, dk, dc


# ---------------------------------------------------------------- global level

def assemble(prob: Problem, rho: np.ndarray):
    """Assemble the global conductivity K, capacity C (both Nn x Nn, CSR) and the
    unit-time load vector f (length Nn) for the design rho (Sec. 2.2).

    The load at time t_j is q_j = q_time[j] * f.
    """
    nx, ny, h = prob.nx, prob.ny, prob.h
    k, c, _, _ = simp(rho, prob.material)
    Ke, Me, fe = element_matrices(h)
    en = element_nodes(nx, ny)
    Nn = prob.Nn
    rows = np.repeat(en, 4, axis=1).reshape(-1)
    cols = np.tile(en, (1, 4)).reshape(-1)
    kv = (k[:, None, None] * Ke[None]).reshape(-1)
    cv = (c[:, None, None] * Me[None]).reshape(-1)
    K = sp.coo_matrix((kv, (rows, cols)), shape=(Nn, Nn)).tocsr()
    C = sp.coo_matrix((cv, (rows, cols)), shape=(Nn, Nn)).tocsr()
    qe = np.ones(prob.Ne) if prob.q_elem is None else np.asarray(prob.q_elem, dtype=np.float64)
    f = np.zeros(Nn)
    np.add.at(f, en.reshape(-1), (qe[:, None] * fe[None]).reshape(-1))
    return K, C, f
