"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds only input generation: the design fields rho, the Dirichlet
node sets, the separable heat-source factors and the workload sizes. It contains
none of the method's arithmetic (no assembly, no time stepping, no objective),
so both the CPU oracle and the CUDA path may consume its arrays without sharing
any computation.

Conventions
-----------
* Grid: ``nx * ny`` square elements of side ``h`` on the rectangle
  ``[0, nx*h] x [0, ny*h]`` (depth 1).  Nodes are numbered row-major,
  ``node = iy * (nx + 1) + ix`` at ``(ix*h, iy*h)``; elements row-major,
  ``e = ey * nx + ex``.
* Every random draw uses ``numpy.random.default_rng(seed)`` in element order
  ``(ey, ex)`` and FP64.

Workloads (sizes follow the paper's test problem of Sec. 5.1 and the scaled
variants used for measurement):

* ``plain32``   32x32, Nt=100, dt=1e-3, rho = 0.5 + U(-0.1, 0.1) seed 0.
* ``oneshot128`` 128x128, Nt=1024 in 32 slices, dt=1/1024, rho ~ U(0.2, 0.8)
  seed 0; the warm-start design is ``clip(rho + U(-0.01, 0.01), 0, 1)`` seed 1000.
* ``diff256``   256x256, Nt=2048 in 64 slices, rho ~ U(0, 1) seed 1.
* ``loop512``   512x512, Nt=4096 in 128 slices, rho = 0.4 uniform.
* ``paper100``  100x100, Nt=480, Table 1 materials, bottom-edge sink,
  q(t) = (1 - t)(1 + cos 50 t)/2 (Eq. 5.1), p = 20.
* ``batch48``   48 designs of uneven size for the batching pattern: design i has side
  (64, 96, 128, 192, 256)[i mod 5], (Nt, Ntau) = ((512, 16), (1024, 32), (2048, 64))[i mod 3]
  (M = 32), dt = 1/Nt, rho ~ U(0.2, 0.8) seed 100 + i (see ``batch48``).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "WORKLOADS", "workload", "rho_plain", "rho_uniform", "rho_warm_perturb",
    "dirichlet_left_centre", "dirichlet_bottom_centre", "dirichlet_none",
    "q_time_paper", "fd_elements", "rho_mirror_y", "batch48", "rho_branches",
]

# Material sets.  "simp_k" is conductivity-only SIMP k = 1e-3 + (1 - 1e-3) rho^3
# with constant unit capacity; "table1" is Table 1 of the paper.
MATERIALS = {
    "simp_k": dict(k0=1.0, kmin=1e-3, pk=3.0, c0=1.0, cmin=1.0, pc=1.0),
    "table1": dict(k0=3.0, kmin=0.03, pk=3.0, c0=1.0, cmin=0.5, pc=2.0),
}

WORKLOADS = {
    "plain32": dict(n=32, Nt=100, Ntau=1, dt=1e-3, p=8.0, material="simp_k", sink="left"),
    "oneshot128": dict(n=128, Nt=1024, Ntau=32, dt=1.0 / 1024, p=8.0, material="simp_k", sink="left"),
    "diff256": dict(n=256, Nt=2048, Ntau=64, dt=1.0 / 2048, p=8.0, material="simp_k", sink="left"),
    "loop512": dict(n=512, Nt=4096, Ntau=128, dt=1.0 / 4096, p=8.0, material="simp_k", sink="left"),
    "paper100": dict(n=100, Nt=480, Ntau=16, dt=1.0 / 480, p=20.0, material="table1", sink="bottom"),
}


def workload(name: str) -> dict:
    """Return a copy of a workload description with its material expanded."""
    w = dict(WORKLOADS[name])
    w["material"] = dict(MATERIALS[w["material"]])
    w["h"] = 1.0 / w["n"]
    return w


def rho_plain(nx: int, ny: int, seed: int = 0, centre: float = 0.5, half: float = 0.1) -> np.ndarray:
    """rho_e = centre + U(-half, half), element order (ey, ex)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(centre - half, centre + half, size=nx * ny).astype(np.float64)


def rho_uniform(nx: int, ny: int, seed: int, lo: float, hi: float) -> np.ndarray:
    """rho_e ~ U(lo, hi), element order (ey, ex)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=nx * ny).astype(np.float64)


def rho_warm_perturb(rho_old: np.ndarray, seed: int = 1000, amp: float = 0.01) -> np.ndarray:
    """The next design of a warm-started iteration: clip(rho_old + U(-amp, amp), 0, 1)."""
    rng = np.random.default_rng(seed)
    return np.clip(rho_old + rng.uniform(-amp, amp, size=rho_old.shape), 0.0, 1.0)


def rho_mirror_y(nx: int, ny: int, seed: int, lo: float = 0.2, hi: float = 0.8) -> np.ndarray:
    """A random design that is mirror-symmetric about the line y = ny*h/2."""
    r = rho_uniform(nx, ny, seed, lo, hi).reshape(ny, nx)
    r = 0.5 * (r + r[::-1, :])
    return r.reshape(-1).copy()


def _node_y(nx: int, ny: int, h: float) -> np.ndarray:
    return (np.arange(ny + 1, dtype=np.float64) * h)[:, None] * np.ones((1, nx + 1))


def _node_x(nx: int, ny: int, h: float) -> np.ndarray:
    return np.ones((ny + 1, 1)) * (np.arange(nx + 1, dtype=np.float64) * h)[None, :]


def dirichlet_left_centre(nx: int, ny: int, h: float, frac: float = 0.1) -> np.ndarray:
    """Sink on the centred ``frac`` of the left edge: nodes with x = 0 and
    |y - L/2| <= frac*L/2 (inclusive, 1e-12 tolerance).  uint8 mask [Nn]."""
    L = ny * h
    x = _node_x(nx, ny, h)
    y = _node_y(nx, ny, h)
    m = (np.abs(x) < 1e-12) & (np.abs(y - 0.5 * L) <= 0.5 * frac * L + 1e-12)
    return m.reshape(-1).astype(np.uint8)


def dirichlet_bottom_centre(nx: int, ny: int, h: float, frac: float = 0.1) -> np.ndarray:
    """Sink on the centred ``frac`` of the bottom edge (Fig. 4 of the paper)."""
    L = nx * h
    x = _node_x(nx, ny, h)
    y = _node_y(nx, ny, h)
    m = (np.abs(y) < 1e-12) & (np.abs(x - 0.5 * L) <= 0.5 * frac * L + 1e-12)
    return m.reshape(-1).astype(np.uint8)


def dirichlet_none(nx: int, ny: int) -> np.ndarray:
    """All-Neumann boundary (used by the separable-eigenmode checks)."""
    return np.zeros((nx + 1) * (ny + 1), dtype=np.uint8)


def q_time_paper(Nt: int, dt: float) -> np.ndarray:
    """Time factor of the paper's load, Eq. 5.1, sampled at t_j = j*dt, j = 0..Nt."""
    t = np.arange(Nt + 1, dtype=np.float64) * dt
    return 0.5 * (1.0 - t) * (1.0 + np.cos(50.0 * t))


def fd_elements(Ne: int, count: int = 32, seed: int = 1) -> np.ndarray:
    """Element indices for finite-difference gradient checks (drawn without replacement)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(Ne, size=count, replace=False))


def batch48() -> list[dict]:
    """The 48 designs of the batching workload: sides cycle through 64, 96, 128, 192, 256
    (10, 10, 10, 9, 9 designs), time grids through (512, 16), (1024, 32), (2048, 64);
    conductivity SIMP, left-centre sink, p = 8, rho ~ U(0.2, 0.8) with seed 100 + index."""
    out = []
    for i in range(48):
        n = (64, 96, 128, 192, 256)[i % 5]
        Nt, Ntau = ((512, 16), (1024, 32), (2048, 64))[i % 3]
        out.append(dict(index=i, n=n, Nt=Nt, Ntau=Ntau, dt=1.0 / Nt, p=8.0, material="simp_k", sink="left",
                        seed=100 + i, rho=rho_uniform(n, n, 100 + i, 0.2, 0.8)))
    return out


def rho_branches(nx: int, ny: int, lo: float = 0.01, hi: float = 0.99) -> np.ndarray:
    """A near-binary design (stand-in for an optimised topology, which is not published): a
    vertical conducting trunk of half-width 0.04 L at x = L/2 over the full height, rising from
    the bottom-edge sink, with three horizontal branches of half-width 0.02 L at y = 0.3, 0.6,
    0.85 L spanning x in [0.1, 0.9] L; rho = hi there and lo elsewhere (element centres)."""
    ey, ex = np.divmod(np.arange(nx * ny), nx)
    x = (ex + 0.5) / nx
    y = (ey + 0.5) / ny
    on = np.abs(x - 0.5) < 0.04
    for yb in (0.3, 0.6, 0.85):
        on |= (np.abs(y - yb) < 0.02) & (x > 0.1) & (x < 0.9)
    return np.where(on, hi, lo).astype(np.float64)

