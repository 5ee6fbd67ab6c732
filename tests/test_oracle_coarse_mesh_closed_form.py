"""Closed-form pins of the coarse-mesh propagators (Sec. 7.3 future work; the readings are those
of oracle/coarse_mesh.py): one G_pri and one G_adj step on a problem that reduces to scalars.

Setting: uniform design, no load, Dirichlet sinks on the whole boundary of an even grid, and the
sine mode v = sin(mx pi x / Lx) sin(my pi y / Ly).
  * Injection takes v to the 2h grid's sine mode v_H of the same (mx, my): node (I, J) is fine
    node (2I, 2J).
  * v_H is an eigenvector of the 2h capacity and conduction matrices: C_H v_H = c mH v_H and
    K_H v_H = k kH v_H, with the 1D eigenvalues h_H (2 + cos t_H) / 3 and 2 (1 - cos t_H) / h_H,
    t_H = m pi / n_H, h_H = 2h (the coarse design is the mean of equal children).
  * Bilinear interpolation of v_H is w = v scaled by cos(mx pi / nx) on odd fine columns and
    by cos(my pi / ny) on odd fine rows (the mean of sin(t (i - 1)) and sin(t (i + 1)) is
    sin(t i) cos t).
  * The transpose of interpolation takes v to (1 + cos(mx pi / nx))(1 + cos(my pi / ny)) v_H.
So G_pri(a v) = a R_H w with R_H = 1 / (1 + dtau mu_H), and its theta increment is the fine-mesh
p-norm of that field.  At p = 2 the adjoint source is a multiple of v, so G_adj(l v) = z w in
closed form, and its g increment combines the element forms w_e^T Ke v_e and w_e^T Me v_e of
the textbook matrices."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import Operator
from oracle.coarse_mesh import CoarseMesh
from tests.problems import make_problem

KE = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
ME1 = np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]]) / 36.0   # times h^2


def _problem(nx, ny, mx, my, Nt, Ntau, p, modified, rho=0.7):
    h = 1.0 / max(nx, ny)
    ix, iy = np.arange(nx + 1), np.arange(ny + 1)
    tx, ty = mx * np.pi / nx, my * np.pi / ny
    v = (np.sin(ty * iy)[:, None] * np.sin(tx * ix)[None, :]).reshape(-1)
    sink = np.zeros((ny + 1, nx + 1), dtype=bool)
    sink[0, :] = sink[-1, :] = sink[:, 0] = sink[:, -1] = True
    v[sink.reshape(-1)] = 0.0
    w = v * (np.where(iy % 2 == 1, np.cos(ty), 1.0)[:, None] * np.where(ix % 2 == 1, np.cos(tx), 1.0)[None, :]).reshape(-1)
    prob = make_problem(nx, ny, Nt=Nt, Ntau=Ntau, dt=0.013, p=p, material="table1", sink=sink.reshape(-1),
                        q_time=np.zeros(Nt + 1), h=h, modified_objective=modified)
    mat = prob.material
    k = mat.kmin + (mat.k0 - mat.kmin) * rho ** mat.pk
    c = mat.cmin + (mat.c0 - mat.cmin) * rho ** mat.pc
    hH, tHx, tHy = 2 * h, mx * np.pi / (nx // 2), my * np.pi / (ny // 2)
    m1x, m1y = hH * (2 + np.cos(tHx)) / 3, hH * (2 + np.cos(tHy)) / 3
    k1x, k1y = 2 * (1 - np.cos(tHx)) / hH, 2 * (1 - np.cos(tHy)) / hH
    return dict(prob=prob, v=v, w=w, h=h, k=k, c=c, mH=m1x * m1y, kH=k1x * m1y + m1x * k1y,
                restrict=(1 + np.cos(tx)) * (1 + np.cos(ty)),
                dk=mat.pk * (mat.k0 - mat.kmin) * rho ** (mat.pk - 1),
                dc=mat.pc * (mat.c0 - mat.cmin) * rho ** (mat.pc - 1), rho=rho)


def _element_forms(S):
    prob = S["prob"]
    nx, ny, h, v, w = prob.nx, prob.ny, S["h"], S["v"], S["w"]
    fk, fm = np.zeros(nx * ny), np.zeros(nx * ny)
    for ey in range(ny):
        for ex in range(nx):
            n0 = ey * (nx + 1) + ex
            idx = [n0, n0 + 1, n0 + nx + 2, n0 + nx + 1]                  # counter-clockwise
            fk[ey * nx + ex] = w[idx] @ KE @ v[idx]
            fm[ey * nx + ex] = h * h * (w[idx] @ ME1 @ v[idx])
    return fk, fm


GRIDS = [(8, 12, 1, 1), (8, 12, 2, 3), (12, 8, 3, 1), (10, 10, 2, 2)]


@pytest.mark.parametrize("nx,ny,mx,my", GRIDS)
@pytest.mark.parametrize("p,modified", [(8.0, False), (2.0, True)])
def test_coarse_mesh_G_pri_step_in_closed_form(nx, ny, mx, my, p, modified):
    Nt, Ntau = 8, 4
    S = _problem(nx, ny, mx, my, Nt, Ntau, p, modified)
    prob = S["prob"]
    cm = CoarseMesh(Operator(prob, np.full(prob.Ne, S["rho"])))
    a, theta_in = 0.8, 0.3
    for s in (0, 2, 3):
        T_new, theta_new = cm.G_pri(s, a * S["v"], theta_in)
        RH = 1.0 / (1.0 + prob.dtau * S["k"] * S["kH"] / (S["c"] * S["mH"]))
        assert np.max(np.abs(T_new - a * RH * S["w"])) < 1e-13 * a
        inc = (a * RH) ** p * np.sum(S["w"] ** p) / (Ntau * prob.Ne)
        expect = theta_in + inc if modified else (theta_in ** p + inc) ** (1 / p)
        assert abs(theta_new - expect) < 1e-13 * expect


@pytest.mark.parametrize("nx,ny,mx,my", GRIDS)
@pytest.mark.parametrize("modified", [True, False])
def test_coarse_mesh_G_adj_step_in_closed_form(nx, ny, mx, my, modified):
    Nt, Ntau, p = 8, 4, 2.0
    M = Nt // Ntau
    S = _problem(nx, ny, mx, my, Nt, Ntau, p, modified)
    prob = S["prob"]
    op = Operator(prob, np.full(prob.Ne, S["rho"]))
    cm = CoarseMesh(op)
    tau = 0.9 ** np.arange(Nt + 1) + 0.05 * np.cos(np.arange(Nt + 1))     # T_hist amplitudes
    T_hist = tau[:, None] * S["v"][None, :]
    Theta = 0.37
    sig = 2.0 / prob.Ne if modified else Theta ** (1 - p) / prob.Ne       # Sec. 7.1 / Eq. 4.6
    fk, fm = _element_forms(S)
    g_in = np.random.default_rng(4).standard_normal(prob.Ne)
    ell = 0.6
    dtau = prob.dtau
    for s in (0, 1, 3):
        kk, kp = M * s + 1, max(M * s + 1 - M, 0)
        lam_new, g_new = cm.G_adj(s, ell * S["v"], g_in, T_hist, Theta)
        cm_dt = S["c"] * S["mH"] / dtau
        z = (cm_dt * ell + sig * tau[kk] * S["restrict"]) / (cm_dt + S["k"] * S["kH"])
        assert np.max(np.abs(lam_new - z * S["w"])) < 1e-12 * abs(z)
        dg = z * (S["dk"] * tau[kk] * fk + S["dc"] * (tau[kk] - tau[kp]) / dtau * fm) / Ntau
        assert np.max(np.abs(g_new - (g_in - dg))) < 1e-12 * np.max(np.abs(dg))
        assert np.max(np.abs(dg)) > 1e-6


def _restrict_by_injection(self, s, lam, g, T_hist, Theta):
    """Planted mistake: the adjoint source taken to the 2h mesh by injection instead of by the
    transpose of interpolation."""
    from oracle.stepping import adjoint_source_scale, sensitivity_term
    prob, opH = self.prob, self.opH
    k, kp = prob.M * s + 1, max(prob.M * s + 1 - prob.M, 0)
    src = adjoint_source_scale(prob, Theta) * T_hist[k] ** (prob.p - 1.0)
    z = opH.solve(prob.dtau, opH.C @ self.R(lam) / prob.dtau + self.R(src))
    lam_new = self.P @ z
    return lam_new, g - sensitivity_term(self.op, lam_new, T_hist[k], T_hist[kp], prob.dtau) / prob.Ntau


def _theta_divisor_Nt(self, s, T, theta):
    """Planted mistake: the coarse theta increment divided by Nt Ne instead of Ntau Ne."""
    from oracle.stepping import accumulate_theta
    prob, opH = self.prob, self.opH
    x = opH.solve(prob.dtau, opH.C @ self.R(T) / prob.dtau + opH.load(prob.M * (s + 1)))
    T_new = self.P @ x
    return T_new, accumulate_theta(prob, theta, T_new, prob.Nt)


@pytest.mark.parametrize("attr,fn", [("G_adj", _restrict_by_injection), ("G_pri", _theta_divisor_Nt)])
def test_a_planted_mistake_fails_the_closed_form(monkeypatch, attr, fn):
    monkeypatch.setattr(CoarseMesh, attr, fn)
    with pytest.raises(AssertionError):
        if attr == "G_pri":
            test_coarse_mesh_G_pri_step_in_closed_form(8, 12, 1, 1, 8.0, False)
        else:
            test_coarse_mesh_G_adj_step_in_closed_form(8, 12, 1, 1, True)
