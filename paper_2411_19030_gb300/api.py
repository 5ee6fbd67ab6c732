"""Python layer over the C ABI: an ``Operator`` handle with one method per entry point,
and the composition of those calls into the sequential pass, the one-shot pass
(Algorithm 3) and k-iteration Parareal.

Every method marshals torch CUDA tensors (FP64, contiguous) into pointers and calls the
library; nothing here computes any step of the method.  Row slices of a tensor are
passed as pointer offsets, so outputs land directly in the caller's state arrays.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _ffi
from ._ffi import (PTG_ADJOINT, PTG_FP32_REFINE, PTG_FP32_REFINE_ALL, PTG_FP64, PTG_OBJ_MODIFIED, PTG_OBJ_POWER_MEAN,
                   PTG_PRIMAL, PTG_SLICES_CHAINED, PTG_SLICES_PARALLEL)

KIND_NAMES = ("fine_primal", "coarse_primal", "correct_primal", "fine_adjoint", "coarse_adjoint", "correct_adjoint")


class PTGError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        super().__init__(f"{what} failed with {_ffi.ERROR_NAMES.get(code, code)}" + (f": {detail}" if detail else ""))


def _lib():
    return _ffi.load()


def _check(rc: int, what: str):
    if rc != 0:
        raise PTGError(rc, what, _lib().ptg_last_error().decode())


def _ptr(t: torch.Tensor | None, device: torch.device | None = None) -> int | None:
    if t is None:
        return None
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("arrays must be contiguous CUDA float64 tensors")
    if device is not None and t.device != device:
        raise ValueError(f"array on {t.device}, operator on {device}")
    return t.data_ptr()


def twolevel_code(v) -> int:
    """The ptg_solve.twolevel value of SolveConfig.twolevel."""
    if isinstance(v, str):
        return {"none": _ffi.PTG_TWOLEVEL_NONE, "additive": _ffi.PTG_TWOLEVEL_ADDITIVE,
                "vcycle": _ffi.PTG_TWOLEVEL_VCYCLE, "threelevel": _ffi.PTG_TWOLEVEL_THREELEVEL}[v]
    return int(v)


@dataclass
class SolveConfig:
    precision: str = "fp64"          # "fp64"; "fp32_refine": fine-step CG in FP32 with FP64 refinement,
    #                                  coarse-step solves in FP64; "fp32_refine_all": every CG in FP32
    rtol: float = 1e-13
    inner_rtol: float = 1e-4
    cg_iters_max: int = 2000
    refine_max: int = 8
    twolevel: bool | int | str = "threelevel"  # preconditioner of the coarse-step solves: "threelevel"
    #                                  (the two-grid cycle whose coarse correction is a two-grid cycle
    #                                  on the 2h level, over aggregates of 2h nodes), "vcycle"
    #                                  (symmetric two-grid cycle with damped-Jacobi smoothing),
    #                                  True / "additive" (D^-1 + P Ac^-1 P^T), False / "none" (Jacobi)
    grid_wide: int = 1               # single FP64 systems over every SM (cooperative grid):
    #                                  0 never, 1 for large grids or when no cluster fits, 2 always
    smooth_steps: int = 0            # V-cycle smoothing: 1 global Jacobi step, k >= 2 slab-local
    #                                  steps, 0 the library default
    coarse_mesh: bool = False        # coarse propagators on the 2h mesh (Sec. 7.3 future work)
    local_steps: int = 0             # FP32 CG without two-level: 1 Jacobi, 2 two slab-local Jacobi
    #                                  steps, 3 the multigrid cycle on streamed fine propagators,
    #                                  0 the library default
    initial_guess: int = 0           # CG start of a step: 1 plain, 2 extrapolated / the neighbouring
    #                                  guess state, 0 the library default (2)
    fine_stream: int = 0             # fine propagators with the CG vectors in global memory, every
    #                                  slice at once: 2 always, 1 never, 0 the library's choice
    coarse_stream: int = 0           # coarse-step solves (G and the correction sweeps) with the CG
    #                                  vectors in global memory and a multigrid V-cycle: 2 always
    #                                  (even grids), 1 never, 0 the library's choice (large grids)


class Operator:
    """One problem (grid, materials, time grid, slices, objective, sink, source) on one GPU.

    material: dict with k0, kmin, pk, c0, cmin, pc (Eq. 2.5-2.6).
    dirichlet: uint8 array [Nn] marking the sink nodes.
    q_elem / q_time: separable source (element density [Ne], time factor [Nt+1]).
    objective: "power_mean" (Theta, Eq. 2.11) or "modified" (Theta~ = Theta^p, Sec. 7.1); every
    theta / g quantity of the passes refers to it (objective_from_modified converts back).
    """

    def __init__(self, nx: int, ny: int, h: float, material: dict, Nt: int, Ntau: int, dt: float, p: float,
                 dirichlet: np.ndarray, q_elem: np.ndarray | None = None, q_time: np.ndarray | None = None,
                 solve: SolveConfig | None = None, device: int | torch.device | None = None,
                 objective: str = "power_mean"):
        lib = _lib()
        solve = solve or SolveConfig()
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else
                           (device.index if isinstance(device, torch.device) else device))
        self.device = dev
        self.nx, self.ny, self.h = nx, ny, h
        self.Nt, self.Ntau, self.dt, self.p = Nt, Ntau, dt, p
        self.material = dict(material)
        self.solve = solve
        self.Nn, self.Ne = (nx + 1) * (ny + 1), nx * ny
        if Nt % Ntau:
            raise ValueError("Ntau must divide Nt")
        self.M = Nt // Ntau
        g = _ffi.ptg_grid(nx, ny, h)
        m = _ffi.ptg_material(material["k0"], material["kmin"], material["pk"],
                              material["c0"], material["cmin"], material["pc"])
        self.objective = objective
        t = _ffi.ptg_time(Nt, Ntau, dt, p, {"power_mean": PTG_OBJ_POWER_MEAN, "modified": PTG_OBJ_MODIFIED}[objective])
        prec = {"fp64": PTG_FP64, "fp32_refine": PTG_FP32_REFINE,
                "fp32_refine_all": PTG_FP32_REFINE_ALL}[solve.precision]
        s = _ffi.ptg_solve(prec, solve.rtol, solve.inner_rtol, solve.cg_iters_max, solve.refine_max,
                           twolevel_code(solve.twolevel), int(solve.grid_wide), int(solve.smooth_steps),
                           int(solve.coarse_mesh), int(solve.local_steps), int(solve.initial_guess),
                           int(solve.fine_stream), int(solve.coarse_stream))
        self._dir = np.ascontiguousarray(dirichlet, dtype=np.uint8).reshape(-1)
        if self._dir.size != self.Nn:
            raise ValueError("dirichlet mask must have (nx+1)(ny+1) entries")
        self._qe = None if q_elem is None else np.ascontiguousarray(q_elem, dtype=np.float64)
        self._qt = None if q_time is None else np.ascontiguousarray(q_time, dtype=np.float64)
        if self._qe is not None and self._qe.size != self.Ne:
            raise ValueError("q_elem must have nx*ny entries")
        if self._qt is not None and self._qt.size != Nt + 1:
            raise ValueError("q_time must have Nt+1 entries")
        handle = ctypes.c_void_p()
        with torch.cuda.device(dev):
            rc = lib.ptg_op_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(t), ctypes.byref(s),
                                   self._dir.ctypes.data,
                                   None if self._qe is None else self._qe.ctypes.data,
                                   None if self._qt is None else self._qt.ctypes.data,
                                   dev.index, ctypes.byref(handle))
        _check(rc, "ptg_op_create")
        self._h = handle

    # ------------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "_h", None):
            _lib().ptg_op_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self, stream=None) -> int:
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return s.cuda_stream

    def zeros(self, *shape) -> torch.Tensor:
        return torch.zeros(*shape, dtype=torch.float64, device=self.device)

    # ------------------------------------------------------------------ entry points
    def assemble(self, rho: torch.Tensor, stream=None):
        """a1: SIMP coefficients and element weights of the design rho [Ne]."""
        if rho.numel() != self.Ne:
            raise ValueError("rho must have nx*ny entries")
        _check(_lib().ptg_fe_assemble_operator(self._h, _ptr(rho, self.device), self._stream(stream)),
               "ptg_fe_assemble_operator")

    def fine_propagate_slices(self, U_T, U_theta, F_T, F_theta, T_hist=None, hist_j0=0, schedule=PTG_SLICES_PARALLEL,
                              s0=0, ns=None, stream=None):
        """a2: F_pri of slices s0..s0+ns-1 (see include/ptg.h)."""
        ns = self.Ntau - s0 if ns is None else ns
        rows = 0 if T_hist is None else T_hist.shape[0]
        _check(_lib().ptg_fine_propagate_slices(self._h, schedule, s0, ns, _ptr(U_T, self.device),
                                                _ptr(U_theta, self.device), _ptr(T_hist, self.device), hist_j0, rows,
                                                _ptr(F_T, self.device), _ptr(F_theta, self.device),
                                                self._stream(stream)), "ptg_fine_propagate_slices")

    def coarse_sweep(self, direction, X_field, X_aux, G_field, G_aux, T_hist=None, Theta=None, stream=None):
        """a3: G of every slice on the guess states X."""
        _check(_lib().ptg_coarse_sweep(self._h, direction, _ptr(X_field, self.device), _ptr(X_aux, self.device),
                                       _ptr(T_hist, self.device), _ptr(Theta, self.device),
                                       _ptr(G_field, self.device), _ptr(G_aux, self.device), self._stream(stream)),
               "ptg_coarse_sweep")

    def coarse_sweep_slices(self, direction, s0, ns, X_field, X_aux, G_field, G_aux, T_hist=None, Theta=None,
                            stream=None):
        """a3 on slices s0..s0+ns-1 only (full-size arrays; only those rows of G are written)."""
        _check(_lib().ptg_coarse_sweep_slices(self._h, direction, s0, ns, _ptr(X_field, self.device),
                                              _ptr(X_aux, self.device), _ptr(T_hist, self.device),
                                              _ptr(Theta, self.device), _ptr(G_field, self.device),
                                              _ptr(G_aux, self.device), self._stream(stream)),
               "ptg_coarse_sweep_slices")

    def coarse_adjoint_split(self, V_lam, V_g, T_hist, H_lam, H_g, S_lam, S_g, s0=0, ns=None, stream=None):
        """a3 (adjoint) as its Theta-free part H and unit-source part S (see include/ptg.h)."""
        ns = self.Ntau - s0 if ns is None else ns
        d = self.device
        _check(_lib().ptg_coarse_adjoint_split(self._h, s0, ns, _ptr(V_lam, d), _ptr(V_g, d), _ptr(T_hist, d),
                                               _ptr(H_lam, d), _ptr(H_g, d), _ptr(S_lam, d), _ptr(S_g, d),
                                               self._stream(stream)), "ptg_coarse_adjoint_split")

    def coarse_adjoint_combine(self, Theta, H_lam, H_g, S_lam, S_g, G_lam, G_g, s0=0, ns=None, stream=None):
        """G = H + c S with the adjoint source scale c of Theta."""
        ns = self.Ntau - s0 if ns is None else ns
        d = self.device
        _check(_lib().ptg_coarse_adjoint_combine(self._h, s0, ns, _ptr(Theta, d), _ptr(H_lam, d), _ptr(H_g, d),
                                                 _ptr(S_lam, d), _ptr(S_g, d), _ptr(G_lam, d), _ptr(G_g, d),
                                                 self._stream(stream)), "ptg_coarse_adjoint_combine")

    def overlap_mode(self) -> int:
        """ptg_op_overlap_ok: 0 the split G_adj may not run beside the forward correction sweep;
        1 it may (and beside F_adj); 2 it may, but F_adj must start after it (shared streaming
        workspace)."""
        if getattr(self, "_overlap_mode", None) is None:
            ok = ctypes.c_int()
            _check(_lib().ptg_op_overlap_ok(self._h, ctypes.byref(ok)), "ptg_op_overlap_ok")
            self._overlap_mode = int(ok.value)
        return self._overlap_mode

    def can_overlap_adjoint_coarse(self) -> bool:
        """Whether the split G_adj may run beside the forward correction sweep (ptg_op_overlap_ok):
        M > 1, fine-mesh G, and neither kind on a cooperative-grid stepper launch."""
        return self.overlap_mode() > 0

    def side_stream(self):
        """Stream of the work that runs beside the forward correction sweep (default priority)."""
        if getattr(self, "_side", None) is None:
            self._side = torch.cuda.Stream(self.device)
        return self._side

    def sweep_stream(self):
        """High-priority stream of the forward correction sweep while work runs beside it: when
        both become ready together, the sweep's thread-block cluster is placed first."""
        if getattr(self, "_sweep", None) is None:
            self._sweep = torch.cuda.Stream(self.device, priority=-100)   # mapped to the highest priority
        return self._sweep

    def parareal_correct(self, direction, F_field, F_aux, G_field, G_aux, X_field, X_aux, T_hist=None, Theta=None,
                         stream=None):
        """a4: the sequential correction sweep (forward or reverse); G_field = G_aux = None is the
        PLT variant (coarse propagators identically zero, Sec. 7)."""
        _check(_lib().ptg_parareal_correct(self._h, direction, _ptr(F_field, self.device), _ptr(F_aux, self.device),
                                           _ptr(G_field, self.device), _ptr(G_aux, self.device),
                                           _ptr(X_field, self.device), _ptr(X_aux, self.device),
                                           _ptr(T_hist, self.device), _ptr(Theta, self.device),
                                           self._stream(stream)), "ptg_parareal_correct")

    def adjoint_sweep(self, T_hist, Theta, V_lam, V_g, F_lam, F_g, hist_j0=0, schedule=PTG_SLICES_PARALLEL, s0=0,
                      ns=None, stream=None):
        """a5: F_adj of slices s0..s0+ns-1."""
        ns = self.Ntau - s0 if ns is None else ns
        _check(_lib().ptg_adjoint_sweep(self._h, schedule, s0, ns, _ptr(T_hist, self.device), hist_j0,
                                        T_hist.shape[0], _ptr(Theta, self.device), _ptr(V_lam, self.device),
                                        _ptr(V_g, self.device), _ptr(F_lam, self.device), _ptr(F_g, self.device),
                                        self._stream(stream)), "ptg_adjoint_sweep")

    def objective_from_modified(self, Theta_mod, grad_mod, Theta, grad, stream=None):
        """Sec. 7.1: Theta = Theta~^(1/p), grad = Theta^(1-p)/p grad~ (outputs may alias inputs)."""
        _check(_lib().ptg_objective_from_modified(self._h, _ptr(Theta_mod, self.device), _ptr(grad_mod, self.device),
                                                  _ptr(Theta, self.device), _ptr(grad, self.device),
                                                  self._stream(stream)), "ptg_objective_from_modified")

    def sensitivities(self, lam_hist, j0, j1, T_hist, grad, hist_j0=0, stream=None):
        """a6: grad += -(1/Nt) sum_j lambda_j^T dR_j/drho (Eq. 4.7)."""
        _check(_lib().ptg_sensitivities(self._h, _ptr(lam_hist, self.device), j0, j1, _ptr(T_hist, self.device),
                                        hist_j0, T_hist.shape[0], _ptr(grad, self.device), self._stream(stream)),
               "ptg_sensitivities")

    def stats(self) -> dict:
        st = _ffi.ptg_stats()
        _check(_lib().ptg_get_stats(self._h, ctypes.byref(st)), "ptg_get_stats")
        out = {}
        for k, _ in _ffi.ptg_stats._fields_:
            if k == "reserved":
                continue
            v = getattr(st, k)
            out[k] = list(v) if k.startswith("kind_") else v
        out["by_kind"] = {name: dict(solves=out["kind_solves"][i], cg_iters=out["kind_cg_iters"][i],
                                     refinements=out["kind_refinements"][i]) for i, name in enumerate(KIND_NAMES)}
        return out

    def set_wait_limit(self, polls: int):
        """Bound of the grid-barrier waits of cooperative-grid launches (0: the default)."""
        _check(_lib().ptg_op_set_wait_limit(self._h, int(polls)), "ptg_op_set_wait_limit")

    def reset_stats(self, stream=None):
        _check(_lib().ptg_reset_stats(self._h, self._stream(stream)), "ptg_reset_stats")

    def plan(self, kind: int, ntasks: int) -> dict:
        cs, nt, ng, mac = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib().ptg_op_get_plan(self._h, kind, ntasks, ctypes.byref(cs), ctypes.byref(nt), ctypes.byref(ng),
                                      ctypes.byref(mac)), "ptg_op_get_plan")
        return dict(cs=cs.value, nthreads=nt.value, ng=ng.value, max_active_clusters=mac.value)

    def set_multigrid(self, solo_rows: int = 0, coarse_steps: int = 0, fused: int = -1):
        """Tune the multigrid cycle of the streamed solves (ptg_op_set_multigrid; 0 / -1 restore
        the defaults)."""
        _check(_lib().ptg_op_set_multigrid(self._h, solo_rows, coarse_steps, fused), "ptg_op_set_multigrid")

    def set_plan(self, kind: int, cs: int, ng: int = 1):
        """Force the cluster size and groups per thread of one task kind (cs = 0 clears it)."""
        _check(_lib().ptg_op_set_plan(self._h, kind, cs, ng), "ptg_op_set_plan")
        self._overlap_mode = None         # the plans decide it


# ---------------------------------------------------------------------- state buffers

class PassBuffers:
    """Device arrays of one pass: the history, the fine / coarse slice results and the
    coarse states of the warm start (old) and of the result (new)."""

    def __init__(self, op: Operator, with_history: bool = True):
        Nt, Ntau, Nn, Ne = op.Nt, op.Ntau, op.Nn, op.Ne
        z = op.zeros
        self.T_hist = z(Nt + 1, Nn) if with_history else None
        self.F_T, self.F_th, self.G_T, self.G_th = z(Ntau, Nn), z(Ntau), z(Ntau, Nn), z(Ntau)
        self.F_l, self.F_g, self.G_l, self.G_g = z(Ntau, Nn), z(Ntau, Ne), z(Ntau, Nn), z(Ntau, Ne)
        self.U_T, self.U_th = z(Ntau + 1, Nn), z(Ntau + 1)          # current coarse states
        self.V_l, self.V_g = z(Ntau + 1, Nn), z(Ntau + 1, Ne)
        self.U_T_new, self.U_th_new = z(Ntau + 1, Nn), z(Ntau + 1)
        self.V_l_new, self.V_g_new = z(Ntau + 1, Nn), z(Ntau + 1, Ne)

    def split_parts(self):
        """The two parts of the adjoint coarse propagator (allocated on first use)."""
        if getattr(self, "H_l", None) is None:
            z = torch.zeros_like
            self.H_l, self.H_g, self.S_l, self.S_g = z(self.G_l), z(self.G_g), z(self.G_l), z(self.G_g)
        return self.H_l, self.H_g, self.S_l, self.S_g

    def swap(self):
        """Make the pass result the warm start of the next pass."""
        self.U_T, self.U_T_new = self.U_T_new, self.U_T
        self.U_th, self.U_th_new = self.U_th_new, self.U_th
        self.V_l, self.V_l_new = self.V_l_new, self.V_l
        self.V_g, self.V_g_new = self.V_g_new, self.V_g


def sequential_pass(op: Operator, buf: PassBuffers, T0: torch.Tensor | None = None, stream=None):
    """Initialisation of Alg. 3: sequential primal (H_pri applied Nt times, full history) and
    sequential adjoint (H_adj applied Nt times), with the coarse checkpoints of both.
    On return buf.U_* / buf.V_* hold (T_{Mn}, theta_{Mn}) and (lambda_{Mn+1}, g_{Mn+1}),
    Theta is buf.U_th[Ntau] and the gradient g_1 is buf.V_g[0]."""
    if T0 is None:
        buf.U_T[0].zero_()
    else:
        buf.U_T[0].copy_(T0)
    buf.U_th[0].zero_()
    op.fine_propagate_slices(buf.U_T, buf.U_th, buf.U_T[1:], buf.U_th[1:], T_hist=buf.T_hist,
                             schedule=PTG_SLICES_CHAINED, stream=stream)
    Theta = buf.U_th[op.Ntau:op.Ntau + 1]
    buf.V_l[op.Ntau].zero_()
    buf.V_g[op.Ntau].zero_()
    op.adjoint_sweep(buf.T_hist, Theta, buf.V_l, buf.V_g, buf.V_l, buf.V_g, schedule=PTG_SLICES_CHAINED,
                     stream=stream)
    return Theta, buf.V_g[0]


def oneshot_pass(op: Operator, buf: PassBuffers, stream=None, plt: bool = False, overlap: bool | None = None):
    """Iteration body of Alg. 3: one modified forward Parareal iteration and one reverse vanilla
    Parareal iteration from the warm start (buf.U_*, buf.V_*).  The corrected states go to
    buf.U_*_new / buf.V_*_new, the history to buf.T_hist; returns (Theta, grad) views.
    plt=True: the coarse propagators are identically zero (Sec. 7): no coarse sweep, and the
    corrections copy the fine results (buf.G_* are left untouched).
    overlap (default: whenever op.can_overlap_adjoint_coarse()): the adjoint coarse propagators
    run as their Theta-free and unit-source parts on a second stream beside the forward
    correction sweep, which occupies one thread-block cluster, and are combined once Theta is
    known (G_adj is affine in the source scale of Eq. 4.6)."""
    if overlap is None:
        overlap = not plt and op.can_overlap_adjoint_coarse()
    if overlap and not plt:
        return _oneshot_pass_overlapped(op, buf, stream)
    Ntau = op.Ntau
    # primal: F and G of every slice on the guess, then the sequential correction
    op.fine_propagate_slices(buf.U_T, buf.U_th, buf.F_T, buf.F_th, T_hist=buf.T_hist, stream=stream)
    if not plt:
        op.coarse_sweep(PTG_PRIMAL, buf.U_T, buf.U_th, buf.G_T, buf.G_th, stream=stream)
    buf.U_T_new[0].copy_(buf.U_T[0])
    buf.U_th_new[0].copy_(buf.U_th[0])
    op.parareal_correct(PTG_PRIMAL, buf.F_T, buf.F_th, None if plt else buf.G_T, None if plt else buf.G_th,
                        buf.U_T_new, buf.U_th_new, T_hist=buf.T_hist, stream=stream)
    Theta = buf.U_th_new[Ntau:Ntau + 1]
    # adjoint: F and G of every slice on the guess, then the reverse correction
    op.adjoint_sweep(buf.T_hist, Theta, buf.V_l, buf.V_g, buf.F_l, buf.F_g, stream=stream)
    if not plt:
        op.coarse_sweep(PTG_ADJOINT, buf.V_l, buf.V_g, buf.G_l, buf.G_g, T_hist=buf.T_hist, Theta=Theta,
                        stream=stream)
    op.parareal_correct(PTG_ADJOINT, buf.F_l, buf.F_g, None if plt else buf.G_l, None if plt else buf.G_g,
                        buf.V_l_new, buf.V_g_new, T_hist=buf.T_hist, Theta=Theta, stream=stream)
    return Theta, buf.V_g_new[0]


def _oneshot_pass_overlapped(op: Operator, buf: PassBuffers, stream=None):
    """oneshot_pass with the split adjoint coarse propagators beside the forward sweep.  The sweep
    runs on a high-priority stream, so that when the fine and coarse primal launches end, its
    single cluster is placed before the parts fill the rest of the GPU."""
    Ntau = op.Ntau
    main = stream if stream is not None else torch.cuda.current_stream(op.device)
    side, hi = op.side_stream(), op.sweep_stream()
    H_l, H_g, S_l, S_g = buf.split_parts()
    with torch.cuda.stream(main):
        buf.U_T_new[0].copy_(buf.U_T[0])
        buf.U_th_new[0].copy_(buf.U_th[0])
    op.fine_propagate_slices(buf.U_T, buf.U_th, buf.F_T, buf.F_th, T_hist=buf.T_hist, stream=main)
    op.coarse_sweep(PTG_PRIMAL, buf.U_T, buf.U_th, buf.G_T, buf.G_th, stream=main)
    primal_done = torch.cuda.Event()
    primal_done.record(main)
    hi.wait_event(primal_done)
    op.parareal_correct(PTG_PRIMAL, buf.F_T, buf.F_th, buf.G_T, buf.G_th, buf.U_T_new, buf.U_th_new,
                        T_hist=buf.T_hist, stream=hi)
    sweep_done = torch.cuda.Event()
    sweep_done.record(hi)
    side.wait_event(primal_done)
    op.coarse_adjoint_split(buf.V_l, buf.V_g, buf.T_hist, H_l, H_g, S_l, S_g, stream=side)
    parts_done = torch.cuda.Event()
    parts_done.record(side)
    Theta = buf.U_th_new[Ntau:Ntau + 1]
    main.wait_event(sweep_done)
    if op.overlap_mode() == 2:            # streamed parts and F_adj share the streaming workspace
        main.wait_event(parts_done)
    op.adjoint_sweep(buf.T_hist, Theta, buf.V_l, buf.V_g, buf.F_l, buf.F_g, stream=main)
    main.wait_event(parts_done)
    op.coarse_adjoint_combine(Theta, H_l, H_g, S_l, S_g, buf.G_l, buf.G_g, stream=main)
    op.parareal_correct(PTG_ADJOINT, buf.F_l, buf.F_g, buf.G_l, buf.G_g, buf.V_l_new, buf.V_g_new,
                        T_hist=buf.T_hist, Theta=Theta, stream=main)
    return Theta, buf.V_g_new[0]


def parareal_pass(op: Operator, buf: PassBuffers, k: int, T0: torch.Tensor | None = None, stream=None):
    """The k-iteration Parareal of the preliminary tests (Sec. 5.2): the coarse initial guess
    u_{s+1}^0 = G_pri(u_s^0), k modified forward Parareal iterations, then the coarse adjoint
    initial guess v_s^0 = G_adj(v_{s+1}^0) on the final history and k reverse iterations.
    Returns (Theta, grad) views; buf.U_* / buf.V_* hold the final coarse states and buf.T_hist
    the final modified-Parareal history.  The initial guesses are correction sweeps with
    F = G_old = 0, so every step runs in the library's kernels."""
    if k < 1:
        raise ValueError("k must be >= 1")
    Ntau = op.Ntau
    for t in (buf.F_T, buf.F_th, buf.G_T, buf.G_th, buf.F_l, buf.F_g, buf.G_l, buf.G_g):
        t.zero_()
    if T0 is None:
        buf.U_T[0].zero_()
    else:
        buf.U_T[0].copy_(T0)
    buf.U_th[0].zero_()
    op.parareal_correct(PTG_PRIMAL, buf.F_T, buf.F_th, buf.G_T, buf.G_th, buf.U_T, buf.U_th, stream=stream)
    for _ in range(k):
        op.fine_propagate_slices(buf.U_T, buf.U_th, buf.F_T, buf.F_th, T_hist=buf.T_hist, stream=stream)
        op.coarse_sweep(PTG_PRIMAL, buf.U_T, buf.U_th, buf.G_T, buf.G_th, stream=stream)
        buf.U_T_new[0].copy_(buf.U_T[0])
        buf.U_th_new[0].copy_(buf.U_th[0])
        op.parareal_correct(PTG_PRIMAL, buf.F_T, buf.F_th, buf.G_T, buf.G_th, buf.U_T_new, buf.U_th_new,
                            T_hist=buf.T_hist, stream=stream)
        buf.U_T, buf.U_T_new = buf.U_T_new, buf.U_T
        buf.U_th, buf.U_th_new = buf.U_th_new, buf.U_th
    Theta = buf.U_th[Ntau:Ntau + 1]
    zl, zg = buf.F_l.zero_(), buf.F_g.zero_()
    buf.G_l.zero_()
    buf.G_g.zero_()
    op.parareal_correct(PTG_ADJOINT, zl, zg, buf.G_l, buf.G_g, buf.V_l, buf.V_g, T_hist=buf.T_hist, Theta=Theta,
                        stream=stream)
    for _ in range(k):
        op.adjoint_sweep(buf.T_hist, Theta, buf.V_l, buf.V_g, buf.F_l, buf.F_g, stream=stream)
        op.coarse_sweep(PTG_ADJOINT, buf.V_l, buf.V_g, buf.G_l, buf.G_g, T_hist=buf.T_hist, Theta=Theta,
                        stream=stream)
        op.parareal_correct(PTG_ADJOINT, buf.F_l, buf.F_g, buf.G_l, buf.G_g, buf.V_l_new, buf.V_g_new,
                            T_hist=buf.T_hist, Theta=Theta, stream=stream)
        buf.V_l, buf.V_l_new = buf.V_l_new, buf.V_l
        buf.V_g, buf.V_g_new = buf.V_g_new, buf.V_g
    return Theta, buf.V_g[0]
