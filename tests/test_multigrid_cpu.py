"""Pins, on the CPU, of the facts the geometric multigrid of the streamed coarse-step solves
rests on (its GPU kernels are checked against the oracle's one-shot pass in test_gpu_mg.py):

* For Q1 elements, the Galerkin product P^T A_h P of bilinear interpolation P from the 2h grid
  is the operator assembled on the 2h grid: the Q1 space on 2h is a subspace of the one on h,
  so the bilinear form restricted to it is the coarse form.  This holds for the conductivity
  and the consistent capacity matrix (Sec. 2.2) of a uniform design, for any step size.
* Hence the largest eigenvalue of D^-1 A, which sets the damped-Jacobi smoother's stability
  (omega lambda_max < 2 with omega = 0.8), keeps the same bound, at most 2.25, on every level.

The matrices come from the oracle's assembly (oracle/fem.py); P and the Galerkin products are
written here."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from oracle.fem import assemble
from tests.problems import make_problem


def bilinear(n: int) -> sp.csr_matrix:
    """P from the (n/2 + 1)^2 nodes of the 2h grid to the (n + 1)^2 nodes of the h grid (row-major
    node order iy * (n + 1) + ix): a fine node takes the mean of the coarse nodes around it."""
    rows, cols, vals = [], [], []
    for x in range(n + 1):
        if x % 2 == 0:
            rows.append(x); cols.append(x // 2); vals.append(1.0)
        else:
            rows += [x, x]; cols += [(x - 1) // 2, (x + 1) // 2]; vals += [0.5, 0.5]
    p1 = sp.csr_matrix((vals, (rows, cols)), shape=(n + 1, n // 2 + 1))
    return sp.kron(p1, p1).tocsr()


def operators(n: int, h: float, rho: float, material: str):
    prob = make_problem(n, Nt=4, dt=0.25, h=h, material=material, sink="left")
    K, C, _ = assemble(prob, np.full(n * n, rho))
    return K.tocsr(), C.tocsr()


def test_galerkin_product_of_bilinear_interpolation_is_the_coarse_q1_operator():
    n, h = 16, 1.0 / 16
    for material, rho in (("simp_k", 0.4), ("table1", 0.7)):
        K, C = operators(n, h, rho, material)
        Kc, Cc = operators(n // 2, 2 * h, rho, material)
        P = bilinear(n)
        for dt in (1e-3, 1.0 / 32, 0.5):
            A = (C / dt + K).tocsr()
            Ac = (Cc / dt + Kc).toarray()
            G = (P.T @ A @ P).toarray()
            assert np.max(np.abs(G - Ac)) <= 1e-12 * np.max(np.abs(Ac)), (material, dt)


def test_jacobi_bound_holds_on_every_galerkin_level():
    n, h = 32, 1.0 / 32
    K, C = operators(n, h, 0.5, "table1")
    for dt in (1.0 / 4096, 1.0 / 128, 1.0):
        A = (C / dt + K).tocsr()
        level, m = A, n
        while m >= 4:
            d = level.diagonal()
            Dm = sp.diags(1.0 / np.sqrt(d))
            lam = spl.eigsh((Dm @ level @ Dm).tocsc(), k=1, which="LA", return_eigenvectors=False)[0]
            assert lam <= 2.25 + 1e-9, (dt, m, lam)
            assert 0.8 * lam < 2.0
            P = bilinear(m)
            level = (P.T @ level @ P).tocsr()
            m //= 2
