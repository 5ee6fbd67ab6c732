"""Pin of k-iteration Parareal (Sec. 4.2 and 5.2: coarse initial guess, then k modified forward
iterations) against the closed form of Gander and Vandewalle (2007, "Analysis of the parareal
time-parallel time-integration method") for a linear problem that reduces to scalars.

On the sine-mode problem of tests/test_oracle_oneshot_closed_form.py (Dirichlet sinks on the
whole boundary, uniform design, no load), F multiplies the mode's amplitude by r^M and G by R
(r = 1/(1 + dt mu), R = 1/(1 + dtau mu)).  From the coarse initial guess beta^0_n = R^n the k-th
iterate at the coarse points is the truncated binomial sum
    beta^k_n = sum_{j=0}^{min(k, n)} C(n, j) (r^M - R)^j R^(n-j),
which equals the fine solution r^(M n) once k >= n.  The modified history holds the uncorrected
F intermediates r^i beta^(k-1)_s between the coarse points (Sec. 4.3), and Theta~ of Sec. 7.1 is
the sum over the slices of the G(iterate k), F(iterate k-1) and G(iterate k-1) increments.  The
reverse iterations that follow (p = 2) obey the same error recursion in matrix form."""
from __future__ import annotations

from math import comb

import numpy as np
import pytest

from oracle import Operator, parareal
from tests.test_oracle_oneshot_closed_form import _setup


@pytest.mark.parametrize("nx,ny,mx,my,Nt,Ntau,p", [(8, 6, 1, 1, 12, 4, 2.0), (7, 9, 2, 1, 15, 5, 8.0),
                                                   (8, 6, 1, 2, 12, 6, 2.0)])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_k_iteration_parareal_matches_the_binomial_closed_form(nx, ny, mx, my, Nt, Ntau, p, k):
    dt, rho = 0.011, 0.7
    S = _setup(nx, ny, mx, my, Nt, Ntau, p, dt, rho, rho)
    prob = S["prob"]
    M = Nt // Ntau
    mu = S["kb"] * S["kh"] / (S["cb"] * S["mh"])
    r, R = 1 / (1 + dt * mu), 1 / (1 + M * dt * mu)
    D = r ** M - R

    def beta(kk, n):
        return sum(comb(n, j) * D ** j * R ** (n - j) for j in range(0, min(kk, n) + 1))

    out = parareal(Operator(prob, np.full(prob.Ne, rho)), k)
    v = S["v"]
    scale = np.max(np.abs(v))
    for n in range(Ntau + 1):
        assert np.max(np.abs(out["U"][0][n] - beta(k, n) * v)) < 1e-12 * scale, n
    for s in range(Ntau):
        for i in range(1, M):
            assert np.max(np.abs(out["T_hist"][M * s + i] - r ** i * beta(k - 1, s) * v)) < 1e-12 * scale
    Pp, Ne = float(np.sum(np.abs(v) ** p)), prob.Ne
    Theta = sum(Pp / Ne * ((R * beta(k, s)) ** p / Ntau
                           + sum((r ** i * beta(k - 1, s)) ** p for i in range(1, M + 1)) / Nt
                           - (R * beta(k - 1, s)) ** p / Ntau) for s in range(Ntau))
    assert abs(out["Theta"] - Theta) < 1e-12 * Theta
    # after k >= n iterations the coarse point n holds the fine solution
    for n in range(min(k, Ntau) + 1):
        assert abs(beta(k, n) - r ** (M * n)) < 1e-14
    if k < Ntau:
        assert abs(beta(k, Ntau) - r ** (M * Ntau)) > 1e-8 * r ** (M * Ntau)


@pytest.mark.parametrize("nx,ny,mx,my,Nt,Ntau", [(8, 6, 1, 1, 12, 4), (8, 6, 2, 1, 15, 5), (7, 9, 1, 2, 12, 6)])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_k_iteration_reverse_parareal_matches_the_matrix_form(nx, ny, mx, my, Nt, Ntau, k):
    """The reverse iterations (Sec. 4.4, Eq. 4.10) at p = 2 with the objective of Sec. 7.1: on the
    mode every adjoint propagator is affine, G(x) = R x + a_s and F(x) = r^M x + b_s, with the
    sources of the final primal history.  The correction cancels a_s, so the error against the
    fixed point l*_s = r^M l*_(s+1) + b_s obeys e^(i+1) = (I - R S)^(-1) (r^M - R) S e^i
    (S the shift s -> s + 1), from the coarse initial guess l^0_s = R l^0_(s+1) + a_s."""
    dt, rho, p = 0.011, 0.7, 2.0
    S = _setup(nx, ny, mx, my, Nt, Ntau, p, dt, rho, rho)
    prob = S["prob"]
    M = Nt // Ntau
    mu = S["kb"] * S["kh"] / (S["cb"] * S["mh"])
    r, R = 1 / (1 + dt * mu), 1 / (1 + M * dt * mu)
    D = r ** M - R

    def beta(kk, n):
        return sum(comb(n, j) * D ** j * R ** (n - j) for j in range(0, min(kk, n) + 1))

    tau = np.zeros(Nt + 1)                                  # the history after k primal iterations
    tau[0] = 1.0
    for s in range(Ntau):
        for i in range(1, M):
            tau[M * s + i] = r ** i * beta(k - 1, s)
        tau[M * (s + 1)] = beta(k, s + 1)
    sig, cm = 2.0 / prob.Ne, S["cb"] * S["mh"]
    a = np.array([R * M * dt * sig * tau[M * s + 1] / cm for s in range(Ntau)])
    b = np.array([sum(r ** (i - M * s) * dt * sig * tau[i] / cm for i in range(M * s + 1, M * (s + 1) + 1))
                  for s in range(Ntau)])
    l0, lstar = np.zeros(Ntau + 1), np.zeros(Ntau + 1)
    for s in range(Ntau - 1, -1, -1):
        l0[s] = R * l0[s + 1] + a[s]
        lstar[s] = r ** M * lstar[s + 1] + b[s]
    shift = np.eye(Ntau + 1, k=1)
    A = np.linalg.solve(np.eye(Ntau + 1) - R * shift, D * shift)
    lam_k = lstar + np.linalg.matrix_power(A, k) @ (l0 - lstar)

    out = parareal(Operator(prob, np.full(prob.Ne, rho)), k)
    v = S["v"]
    scale = np.max(np.abs(lam_k)) * np.max(np.abs(v))
    for s in range(Ntau + 1):
        assert np.max(np.abs(out["V"][0][s] - lam_k[s] * v)) < 1e-11 * scale, s
    if k < Ntau:                                            # not yet at the fixed point
        assert np.max(np.abs(lam_k - lstar)) > 1e-6 * np.max(np.abs(lstar))
