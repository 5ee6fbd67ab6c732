"""Test-side helpers that build oracle problems from the seeded workloads."""
from __future__ import annotations

import numpy as np

import workloads as W
from oracle import Material, Problem


def make_problem(nx, ny=None, *, Nt, Ntau=1, dt=None, p=8.0, material="simp_k", sink="left",
                 q_elem=None, q_time=None, T0=None, h=None, modified_objective=False) -> Problem:
    ny = nx if ny is None else ny
    h = 1.0 / max(nx, ny) if h is None else h
    dt = 1.0 / Nt if dt is None else dt
    mat = Material(**W.MATERIALS[material]) if isinstance(material, str) else material
    if isinstance(sink, np.ndarray):
        dir_mask = sink
    elif sink == "left":
        dir_mask = W.dirichlet_left_centre(nx, ny, h)
    elif sink == "left_wide":
        dir_mask = W.dirichlet_left_centre(nx, ny, h, frac=0.5)
    elif sink == "bottom":
        dir_mask = W.dirichlet_bottom_centre(nx, ny, h)
    elif sink == "none":
        dir_mask = W.dirichlet_none(nx, ny)
    else:
        raise ValueError(sink)
    return Problem(nx=nx, ny=ny, h=h, material=mat, Nt=Nt, dt=dt, Ntau=Ntau, p=p,
                   dirichlet=dir_mask, q_elem=q_elem, q_time=q_time, T0=T0,
                   modified_objective=modified_objective)


def workload_problem(name: str, Ntau=None) -> tuple[Problem, np.ndarray]:
    """The oracle Problem and design rho of a named workload."""
    w = W.workload(name)
    n = w["n"]
    prob = make_problem(n, Nt=w["Nt"], Ntau=w["Ntau"] if Ntau is None else Ntau, dt=w["dt"], p=w["p"],
                        material=Material(**w["material"]), sink=w["sink"],
                        q_time=W.q_time_paper(w["Nt"], w["dt"]) if name == "paper100" else None)
    if name == "plain32":
        rho = W.rho_plain(n, n, seed=0)
    elif name == "oneshot128":
        rho = W.rho_uniform(n, n, 0, 0.2, 0.8)
    elif name == "diff256":
        rho = W.rho_uniform(n, n, 1, 0.0, 1.0)
    else:
        rho = np.full(n * n, 0.4 if name == "loop512" else 0.3)
    return prob, rho
