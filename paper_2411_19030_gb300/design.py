"""The one-shot design loop of Alg. 3 around the pass: the design parametrisation of
Sec. 2.1 (density filter and threshold projection, ``DesignMap`` over ``ptg_design_*``), the
area constraint of Sec. 3, and the Method of Moving Asymptotes on the host (``MMAUpdate``
over ``ptg_mma_*``).

``OneShotLoop.run`` performs the optimisation: the first design iteration solves the state
and adjoint by sequential time stepping (the initialisation of Alg. 3), every later one by
one modified forward and one reverse Parareal iteration warm-started from the previous
iteration's coarse states (the iteration body of Alg. 3).  Each iteration maps chi to rho on
the device, assembles, runs the pass, applies the chain rule on the device, copies the
objective, the area fraction and the two gradients to the host and lets MMA produce the next
chi.  The objective passed to MMA is Theta / Theta_1 (scaled by the first iteration's value).
"""
from __future__ import annotations

import ctypes
import time

import numpy as np
import torch

from .api import Operator, PassBuffers, _check, _lib, oneshot_pass, sequential_pass


class DesignMap:
    """chi -> rho = P(H chi) and the chain rule back to chi, on the device (FP64)."""

    def __init__(self, nx: int, ny: int, h: float, r_fil: float, beta: float, eta: float = 0.5,
                 device: int | torch.device | None = None):
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else
                           (device.index if isinstance(device, torch.device) else device))
        self.device = dev
        self.Ne = nx * ny
        h_ = ctypes.c_void_p()
        _check(_lib().ptg_design_create(nx, ny, h, r_fil, beta, eta, dev.index, ctypes.byref(h_)), "ptg_design_create")
        self._h = h_

    def close(self):
        if getattr(self, "_h", None):
            _lib().ptg_design_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _s(self, stream):
        return (stream or torch.cuda.current_stream(self.device)).cuda_stream

    def forward(self, chi, rho, dproj, stream=None):
        _check(_lib().ptg_design_forward(self._h, chi.data_ptr(), rho.data_ptr(), dproj.data_ptr(), self._s(stream)),
               "ptg_design_forward")

    def backward(self, dproj, df_drho, out, stream=None):
        """out = H^T (dproj * df_drho); df_drho None: the gradient of the area fraction."""
        _check(_lib().ptg_design_backward(self._h, dproj.data_ptr(), None if df_drho is None else df_drho.data_ptr(),
                                          out.data_ptr(), self._s(stream)), "ptg_design_backward")

    def volume(self, rho, out, stream=None):
        _check(_lib().ptg_design_volume(self._h, rho.data_ptr(), out.data_ptr(), self._s(stream)),
               "ptg_design_volume")


class MMAUpdate:
    """The Method of Moving Asymptotes on the host (min f0 s.t. f1 <= 0, box bounds)."""

    def __init__(self, n: int, x_min: float = 0.0, x_max: float = 1.0, move: float = 0.2):
        self.n = n
        h = ctypes.c_void_p()
        _check(_lib().ptg_mma_create(n, x_min, x_max, move, ctypes.byref(h)), "ptg_mma_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib().ptg_mma_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, x: np.ndarray, f0: float, df0: np.ndarray, f1: float, df1: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        df0 = np.ascontiguousarray(df0, dtype=np.float64)
        df1 = np.ascontiguousarray(df1, dtype=np.float64)
        out = np.empty_like(x)
        _check(_lib().ptg_mma_update(self._h, x.ctypes.data, float(f0), df0.ctypes.data, float(f1), df1.ctypes.data,
                                     out.ctypes.data), "ptg_mma_update")
        return out

    def get_state(self) -> dict:
        """The update count and the last two iterates and asymptotes (host copies)."""
        k = ctypes.c_longlong()
        arrs = {name: np.empty(self.n) for name in ("x1", "x2", "L", "U")}
        _check(_lib().ptg_mma_get_state(self._h, ctypes.byref(k), *(a.ctypes.data for a in arrs.values())),
               "ptg_mma_get_state")
        return dict(k=k.value, **arrs)

    def set_state(self, st: dict):
        arrs = [np.ascontiguousarray(st[name], dtype=np.float64) for name in ("x1", "x2", "L", "U")]
        if any(a.size != self.n for a in arrs):
            raise ValueError("MMA state of another size")
        _check(_lib().ptg_mma_set_state(self._h, int(st["k"]), *(a.ctypes.data for a in arrs)), "ptg_mma_set_state")


class OneShotLoop:
    """Alg. 3 for one design: ``op`` holds the problem (its precision is the pass's), ``design``
    the filter and projection, a_max the area fraction bound.  ``true_op`` (optional, e.g. FP64)
    recomputes the true objective of the current design by a sequential pass every
    ``true_every`` iterations for the convergence history (outside the timed iteration)."""

    def __init__(self, op: Operator, design: DesignMap, a_max: float, move: float = 0.2,
                 true_op: Operator | None = None):
        self.op, self.design, self.a_max = op, design, a_max
        self.buf = PassBuffers(op)
        self.mma = MMAUpdate(op.Ne, 0.0, 1.0, move)
        self.true_op = true_op
        z = op.zeros
        self.chi_d, self.rho, self.dproj = z(op.Ne), z(op.Ne), z(op.Ne)
        self.g_chi, self.v_chi, self.vol = z(op.Ne), z(op.Ne), z(1)
        self.theta1 = None

    def iterate(self, chi: np.ndarray, first: bool, stream=None) -> dict:
        """One design iteration from chi (host); returns the new chi and the iteration's values."""
        op, des, buf = self.op, self.design, self.buf
        self.chi_d.copy_(torch.from_numpy(chi), non_blocking=False)
        des.forward(self.chi_d, self.rho, self.dproj, stream)
        op.assemble(self.rho, stream=stream)
        if first:
            Theta, g_rho = sequential_pass(op, buf, stream=stream)
        else:
            Theta, g_rho = oneshot_pass(op, buf, stream=stream)
        des.backward(self.dproj, g_rho, self.g_chi, stream)
        des.volume(self.rho, self.vol, stream)
        des.backward(self.dproj, None, self.v_chi, stream)
        torch.cuda.synchronize(op.device)
        theta = float(Theta.item())
        if self.theta1 is None:
            self.theta1 = theta
        vol = float(self.vol.item())
        g = self.g_chi.cpu().numpy() / self.theta1
        v = self.v_chi.cpu().numpy()
        chi_new = self.mma.update(chi, theta / self.theta1, g, vol - self.a_max, v)
        if not first:
            buf.swap()        # this iteration's coarse states warm-start the next one
        return dict(chi=chi_new, Theta=theta, volume=vol)

    def true_objective(self) -> float:
        """Theta of the current rho by a sequential pass of true_op."""
        top = self.true_op
        tb = PassBuffers(top, with_history=True)
        top.assemble(self.rho)
        Theta, _ = sequential_pass(top, tb)
        return float(Theta.item())

    # ------------------------------------------------------------------ save / resume
    def save(self, path: str, chi: np.ndarray, iteration: int):
        """Write everything the loop carries from one design iteration to the next: the design
        variable chi to be evaluated next, the number of iterations done, the objective scale
        Theta_1, the coarse states of the warm start (u^old = (T, theta), v^old = (lambda, g)),
        and the MMA state; plus the problem sizes, which load() checks."""
        torch.cuda.synchronize(self.op.device)
        op, b = self.op, self.buf
        np.savez(path, chi=np.asarray(chi, dtype=np.float64), iteration=int(iteration),
                 theta1=np.nan if self.theta1 is None else self.theta1,
                 U_T=b.U_T.cpu().numpy(), U_th=b.U_th.cpu().numpy(), V_l=b.V_l.cpu().numpy(),
                 V_g=b.V_g.cpu().numpy(), sizes=np.array([op.nx, op.ny, op.Nt, op.Ntau]),
                 **{"mma_" + k: v for k, v in self.mma.get_state().items()})

    def load(self, path: str) -> tuple[np.ndarray, int]:
        """Restore a state written by save() into this loop (same problem sizes); returns
        (chi, iterations done) to pass to run(..., start=iterations done)."""
        d = np.load(path)
        op, b = self.op, self.buf
        if list(d["sizes"]) != [op.nx, op.ny, op.Nt, op.Ntau]:
            raise ValueError(f"saved state is for sizes {list(d['sizes'])}, not {[op.nx, op.ny, op.Nt, op.Ntau]}")
        for t, name in ((b.U_T, "U_T"), (b.U_th, "U_th"), (b.V_l, "V_l"), (b.V_g, "V_g")):
            t.copy_(torch.from_numpy(d[name]))
        th1 = float(d["theta1"])
        self.theta1 = None if np.isnan(th1) else th1
        self.mma.set_state({k: d["mma_" + k] for k in ("k", "x1", "x2", "L", "U")})
        torch.cuda.synchronize(op.device)
        return d["chi"].copy(), int(d["iteration"])

    def run(self, chi0: np.ndarray, iterations: int, true_every: int = 0, start: int = 0) -> dict:
        """Design iterations start .. iterations-1 from chi0 (iteration 0 is the sequential one;
        a resumed loop passes the state's iteration count as start)."""
        chi = np.ascontiguousarray(chi0, dtype=np.float64)
        hist = dict(Theta=[], volume=[], ms=[], true_Theta={})
        for k in range(start, iterations):
            torch.cuda.synchronize(self.op.device)
            t0 = time.perf_counter()
            out = self.iterate(chi, first=(k == 0))
            hist["ms"].append(1e3 * (time.perf_counter() - t0))
            chi = out["chi"]
            hist["Theta"].append(out["Theta"])
            hist["volume"].append(out["volume"])
            if self.true_op is not None and true_every and ((k + 1) % true_every == 0 or k + 1 == iterations):
                hist["true_Theta"][k] = self.true_objective()
        hist["chi"] = chi
        return hist
