"""Several designs advanced together (the batching pattern): ``Batch`` wraps the
``ptg_batch_*`` entry points, ``autotune`` picks each phase's launch plan by timing the
candidate plans on the batch itself, and ``Batch.capture`` records assembly plus a whole
one-shot pass of every design in one CUDA graph.

Each phase of a pass (fine primal, coarse primal, primal correction, fine adjoint, coarse
adjoint, adjoint correction) is one persistent launch over all designs and slices; the
batch owns each design's device buffers, exposed as torch tensors by ``Batch.buffers``.
"""
from __future__ import annotations

import ctypes

import torch

from . import _ffi
from ._ffi import PTG_PARAREAL, PTG_PLT
from .api import Operator, _check, _lib

PHASES = ("fine_primal", "coarse_primal", "correct_primal", "fine_adjoint", "coarse_adjoint", "correct_adjoint",
          "sequential_primal", "sequential_adjoint")


def device_view(ptr: int, shape, device) -> torch.Tensor:
    """A torch tensor over library-owned device memory (FP64, contiguous, no copy); the
    library frees the memory, so the view must not outlive the batch."""
    n = 1
    for s in shape:
        n *= s

    class _CudaArray:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False), "version": 3,
                                    "strides": None}

    return torch.as_tensor(_CudaArray(), device=device).view(*shape)


class Batch:
    """A batch of designs; ``ops`` are ``Operator``s of one precision on one device (grid sizes,
    time grids and slice counts may differ)."""

    def __init__(self, ops: list[Operator]):
        self.ops = list(ops)
        self.device = ops[0].device
        arr = (ctypes.c_void_p * len(ops))(*[op._h.value for op in ops])
        h = ctypes.c_void_p()
        _check(_lib().ptg_batch_create(arr, len(ops), ctypes.byref(h)), "ptg_batch_create")
        self._h = h
        self.graph = None
        self._views = [self._make_views(d) for d in range(len(ops))]

    def close(self):
        if getattr(self, "_h", None):
            self.graph = None
            self._views = []
            _lib().ptg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _make_views(self, d: int) -> dict:
        b = _ffi.ptg_pass_buffers()
        _check(_lib().ptg_batch_buffers(self._h, d, ctypes.byref(b)), "ptg_batch_buffers")
        op = self.ops[d]
        T, Nn, Ne, Nt = op.Ntau, op.Nn, op.Ne, op.Nt
        shapes = {"T_hist": (Nt + 1, Nn), "U_T": (T + 1, Nn), "U_theta": (T + 1,), "V_lam": (T + 1, Nn),
                  "V_g": (T + 1, Ne), "U_T_new": (T + 1, Nn), "U_theta_new": (T + 1,), "V_lam_new": (T + 1, Nn),
                  "V_g_new": (T + 1, Ne), "F_T": (T, Nn), "F_theta": (T,), "G_T": (T, Nn), "G_theta": (T,),
                  "F_lam": (T, Nn), "F_g": (T, Ne), "G_lam": (T, Nn), "G_g": (T, Ne), "rho": (Ne,)}
        return {k: device_view(getattr(b, k), v, self.device) for k, v in shapes.items()}

    def buffers(self, d: int) -> dict:
        """Torch views of design d's batch-owned buffers (valid while the batch lives)."""
        return self._views[d]

    def _stream(self, stream=None) -> int:
        return (stream if stream is not None else torch.cuda.current_stream(self.device)).cuda_stream

    def assemble(self, stream=None):
        _check(_lib().ptg_batch_assemble(self._h, self._stream(stream)), "ptg_batch_assemble")

    def sequential_pass(self, stream=None):
        _check(_lib().ptg_batch_sequential_pass(self._h, self._stream(stream)), "ptg_batch_sequential_pass")

    def oneshot_pass(self, stream=None, plt: bool = False):
        """The iteration body of Alg. 3 for every design; plt=True: coarse propagators
        identically zero (Sec. 7)."""
        _check(_lib().ptg_batch_oneshot_pass(self._h, PTG_PLT if plt else PTG_PARAREAL, self._stream(stream)),
               "ptg_batch_oneshot_pass")

    def commit(self, stream=None):
        _check(_lib().ptg_batch_commit(self._h, self._stream(stream)), "ptg_batch_commit")

    def run_phase(self, phase: int, stream=None):
        _check(_lib().ptg_batch_run_phase(self._h, phase, self._stream(stream)), "ptg_batch_run_phase")

    def set_plan(self, phase: int, cs: int, ng: int, nthreads: int):
        _check(_lib().ptg_batch_set_plan(self._h, phase, cs, ng, nthreads), "ptg_batch_set_plan")

    def own_path(self, d: int) -> bool:
        """Whether design d runs the pass phases through its op's own launches (streamed
        coarse-step solves) rather than in the persistent launches."""
        own = ctypes.c_int()
        _check(_lib().ptg_batch_design_path(self._h, d, ctypes.byref(own)), "ptg_batch_design_path")
        return bool(own.value)

    def plan(self, phase: int) -> dict:
        cs, ng, nt, ncl = (ctypes.c_int() for _ in range(4))
        _check(_lib().ptg_batch_get_plan(self._h, phase, ctypes.byref(cs), ctypes.byref(ng), ctypes.byref(nt),
                                         ctypes.byref(ncl)), "ptg_batch_get_plan")
        return dict(cs=cs.value, ng=ng.value, nthreads=nt.value, nclusters=ncl.value)

    def capture(self) -> torch.cuda.CUDAGraph:
        """Record assembly + one-shot pass of every design into a CUDA graph; ``replay()`` runs
        it.  The plans of all six phases are fixed first, so nothing is uploaded while the
        stream is being captured."""
        for ph in range(6):
            self.plan(ph)
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):          # one uncaptured pass on the capture stream
            self.assemble(s)
            self.oneshot_pass(s)
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.assemble(s)
            self.oneshot_pass(s)
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()


def candidate_plans(batch: Batch):
    """Valid (cluster size, groups per thread, threads per CTA) candidates: for every cluster
    size and NG the smallest block that holds the slab of the largest design of the persistent
    launches, and twice that."""
    out = []
    ops = [op for d, op in enumerate(batch.ops) if not batch.own_path(d)] or batch.ops
    for cs in (16, 8, 4, 2):
        rows = [(op.ny + 1 + cs - 1) // cs for op in ops]
        if min(rows) < 2:
            continue
        groups = max(r * (((op.nx + 3 + 3) // 4 * 4) // 4) for r, op in zip(rows, ops))
        for ng in range(1, 7):
            nt = -(-groups // ng)
            nt = -(-nt // 32) * 32
            for t in (nt, 2 * nt):
                if t <= 512:
                    out.append((cs, ng, t))
    return out


def autotune(batch: Batch, phases=range(6), reps: int = 2, verbose: bool = False) -> dict:
    """Pick each phase's plan by timing every candidate of ``candidate_plans`` on the batch's
    current buffers (one full pass first makes every phase's inputs current; each candidate
    then re-runs its phase alone, which is idempotent).  The fastest plan is installed.
    Returns {phase name: ((cs, ng, nthreads), ms)}."""
    stream = torch.cuda.current_stream(batch.device)
    batch.oneshot_pass()
    result = {}
    for ph in phases:
        best = None
        for cs, ng, nt in candidate_plans(batch):
            if _lib().ptg_batch_set_plan(batch._h, ph, cs, ng, nt) != 0:
                continue
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            times = []
            for _ in range(reps):
                a.record(stream)
                batch.run_phase(ph)
                b.record(stream)
                b.synchronize()
                times.append(a.elapsed_time(b))
            ms = min(times)
            if verbose:
                print(f"{PHASES[ph]:18s} cs={cs:2d} ng={ng} nthreads={nt:3d}: {ms:8.3f} ms")
            if best is None or ms < best[1]:
                best = ((cs, ng, nt), ms)
        if best is not None:
            batch.set_plan(ph, *best[0])
            result[PHASES[ph]] = best
    return result
