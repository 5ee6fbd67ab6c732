"""Design parametrisation and design update (Sec. 2.1, Sec. 3, Alg. 3): the linear density
filter H, the threshold projection P, the area constraint, their chain rule, and the Method
of Moving Asymptotes for one constraint.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Filter (Sec. 2.1): chi_fil = H chi, a weighted average of the element values within a distance
r_fil of each element centre.  Reading: cone weights w_ij = max(0, r_fil - |c_i - c_j|) over the
element centres c (the classical density filter of the works the paper cites), each row
normalised to sum 1, so H_ij = w_ij / sum_k w_ik.

Projection (Sec. 2.1): chi_phys = P(chi_fil) = (tanh(beta (x - eta)) + tanh(beta eta)) /
(tanh(beta (1 - eta)) + tanh(beta eta)), dP/dx = beta (1 - tanh^2(beta (x - eta))) / (same
denominator).  chi_phys is the element density rho of the SIMP laws.

Area constraint (Sec. 3): sum_e chi_phys,e h^2 <= a_max A, i.e. mean(chi_phys) - a_max <= 0 on a
uniform grid.

Chain rule: for rho = P(H chi), d f / d chi = H^T (P'(H chi) * d f / d rho).

MMA (Svanberg 1987; the paper uses a variant for large beta that it does not give, so the
plain method is used): at the iterate x with objective f0, constraint f1 and their gradients,
  * asymptotes L, U: x -+ 0.5 (x_max - x_min) in the first two iterations, afterwards
    x -+ gamma (x_prev -+ L_prev / U_prev) with gamma = 0.7 if x oscillated, 1.2 if it moved
    the same way twice, 1 otherwise;
  * box alpha = max(x_min, L + 0.1 (x - L), x - move), beta = min(x_max, U - 0.1 (U - x), x + move);
  * convex separable approximations with p_ij = (U_j - x_j)^2 max(0, d_j f_i) and
    q_ij = (x_j - L_j)^2 max(0, -d_j f_i), plus the positive terms 1e-3 |d_j f_i| + 1e-6/(x_max -
    x_min) on both sides so that every approximation is strictly convex;
  * the subproblem min_x sum_j p0j/(U_j - x_j) + q0j/(x_j - L_j) subject to the approximated
    constraint and alpha <= x <= beta, solved through its dual in the single multiplier lam >= 0:
    x_j(lam) minimises (p0j + lam p1j)/(U_j - x) + (q0j + lam q1j)/(x - L_j) on [alpha_j, beta_j],
    x_j = (L_j sqrt(P) + U_j sqrt(Q)) / (sqrt(P) + sqrt(Q)) clipped, with P = p0j + lam p1j,
    Q = q0j + lam q1j; the approximated constraint at x(lam) decreases in lam, so lam = 0 if it
    holds there, otherwise the root found by bisection.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def filter_matrix(nx: int, ny: int, h: float, r_fil: float) -> sp.csr_matrix:
    """H with cone weights over element centres, rows normalised (Sec. 2.1)."""
    Ne = nx * ny
    ey, ex = np.divmod(np.arange(Ne), nx)
    R = int(np.ceil(r_fil / h))
    rows, cols, vals = [], [], []
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            w = r_fil - h * np.hypot(dx, dy)
            if w <= 0:
                continue
            jy, jx = ey + dy, ex + dx
            ok = (jy >= 0) & (jy < ny) & (jx >= 0) & (jx < nx)
            rows.append(np.nonzero(ok)[0])
            cols.append(jy[ok] * nx + jx[ok])
            vals.append(np.full(ok.sum(), w))
    W = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(Ne, Ne))
    s = np.asarray(W.sum(axis=1)).ravel()
    return sp.diags(1.0 / s) @ W


def project(x: np.ndarray, beta: float, eta: float) -> np.ndarray:
    den = np.tanh(beta * (1.0 - eta)) + np.tanh(beta * eta)
    return (np.tanh(beta * (x - eta)) + np.tanh(beta * eta)) / den


def project_derivative(x: np.ndarray, beta: float, eta: float) -> np.ndarray:
    den = np.tanh(beta * (1.0 - eta)) + np.tanh(beta * eta)
    return beta * (1.0 - np.tanh(beta * (x - eta)) ** 2) / den


class Design:
    """chi -> rho = P(H chi) and the chain rule back to chi."""

    def __init__(self, nx: int, ny: int, h: float, r_fil: float, beta: float, eta: float):
        self.H = filter_matrix(nx, ny, h, r_fil)
        self.beta, self.eta = beta, eta
        self.Ne = nx * ny

    def forward(self, chi: np.ndarray):
        xf = self.H @ np.asarray(chi, dtype=np.float64)
        return project(xf, self.beta, self.eta), project_derivative(xf, self.beta, self.eta)

    def backward(self, dproj: np.ndarray, df_drho: np.ndarray) -> np.ndarray:
        return self.H.T @ (dproj * np.asarray(df_drho, dtype=np.float64))

    def volume(self, rho: np.ndarray, a_max: float) -> float:
        return float(np.mean(rho)) - a_max

    def volume_gradient(self, dproj: np.ndarray) -> np.ndarray:
        return self.backward(dproj, np.full(self.Ne, 1.0 / self.Ne))


class MMA:
    """The Method of Moving Asymptotes for min f0 s.t. f1 <= 0, x_min <= x <= x_max."""

    def __init__(self, n: int, x_min: float = 0.0, x_max: float = 1.0, move: float = 0.2):
        self.n, self.x_min, self.x_max, self.move = n, x_min, x_max, move
        self.k = 0
        self.x1 = self.x2 = None     # the previous two iterates
        self.L = self.U = None

    def asymptotes(self, x: np.ndarray):
        span = self.x_max - self.x_min
        if self.k < 2:
            L, U = x - 0.5 * span, x + 0.5 * span
        else:
            s = (x - self.x1) * (self.x1 - self.x2)
            gamma = np.where(s < 0, 0.7, np.where(s > 0, 1.2, 1.0))
            L = x - gamma * (self.x1 - self.L)
            U = x + gamma * (self.U - self.x1)
        return L, U

    @staticmethod
    def _pq(df, x, L, U, span):
        pos, neg = np.maximum(df, 0.0), np.maximum(-df, 0.0)
        reg = 1e-3 * np.abs(df) + 1e-6 / span
        return (U - x) ** 2 * (pos + reg), (x - L) ** 2 * (neg + reg)

    @staticmethod
    def _x_of(lam, p0, q0, p1, q1, L, U, a, b):
        P = p0 + lam * p1
        Q = q0 + lam * q1
        sP, sQ = np.sqrt(P), np.sqrt(Q)
        return np.clip((L * sP + U * sQ) / (sP + sQ), a, b)

    def update(self, x, f0, df0, f1, df1):
        """One MMA step from x; returns the new iterate."""
        x = np.asarray(x, dtype=np.float64)
        span = self.x_max - self.x_min
        L, U = self.asymptotes(x)
        a = np.maximum.reduce([np.full_like(x, self.x_min), L + 0.1 * (x - L), x - self.move])
        b = np.minimum.reduce([np.full_like(x, self.x_max), U - 0.1 * (U - x), x + self.move])
        p0, q0 = self._pq(np.asarray(df0), x, L, U, span)
        p1, q1 = self._pq(np.asarray(df1), x, L, U, span)
        r1 = f1 - np.sum(p1 / (U - x) + q1 / (x - L))

        def g(lam):
            xl = self._x_of(lam, p0, q0, p1, q1, L, U, a, b)
            return float(np.sum(p1 / (U - xl) + q1 / (xl - L)) + r1), xl

        g0, x_new = g(0.0)
        if g0 > 0.0:
            lo, hi = 0.0, 1.0
            while g(hi)[0] > 0.0 and hi < 1e30:
                hi *= 2.0
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if g(mid)[0] > 0.0:
                    lo = mid
                else:
                    hi = mid
                if hi - lo <= 1e-14 * hi:
                    break
            x_new = g(hi)[1]
        self.x2, self.x1 = self.x1, x.copy()
        self.L, self.U = L, U
        self.k += 1
        return x_new


def design_loop(prob, r_fil: float, beta: float, eta: float, a_max: float, chi0, iterations: int,
                move: float = 0.2) -> dict:
    """Alg. 3 for one problem: iteration 1 by sequential time stepping, later iterations by one
    one-shot Parareal pass warm-started from the previous iteration's coarse states; the
    design rho = P(H chi); MMA on (Theta / Theta_1, area fraction - a_max).  Returns the
    objective, area fraction and chi of every iteration."""
    from .parareal import coarse_states_from_sequential, oneshot_pass
    from .stepping import Operator

    des = Design(prob.nx, prob.ny, prob.h, r_fil, beta, eta)
    mma = MMA(prob.nx * prob.ny, 0.0, 1.0, move)
    chi = np.asarray(chi0, dtype=np.float64).copy()
    U = V = None
    theta1 = None
    hist = dict(Theta=[], volume=[], chi=[])
    for k in range(iterations):
        rho, dproj = des.forward(chi)
        op = Operator(prob, rho)
        if k == 0:
            U, V, seq = coarse_states_from_sequential(op)
            Theta, grad = seq["Theta"], seq["grad"]
        else:
            out = oneshot_pass(op, U, V)
            Theta, grad = out["Theta"], out["grad"]
            U, V = out["U"], out["V"]
        if theta1 is None:
            theta1 = Theta
        vol = float(np.mean(rho))
        chi = mma.update(chi, Theta / theta1, des.backward(dproj, grad) / theta1, vol - a_max,
                         des.volume_gradient(dproj))
        hist["Theta"].append(Theta)
        hist["volume"].append(vol)
        hist["chi"].append(chi.copy())
    return hist

