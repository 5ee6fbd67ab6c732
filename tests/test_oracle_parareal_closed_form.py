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
the sum over the slices of the G(iterate k), F(iterate k-1) and G(iterate k-1) increments."""
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
