"""Differentiation of the objective with respect to the design: ``ParaTopoFn``.

Theta(rho) of Eq. 2.11 with the discrete-adjoint gradient of Eq. 4.4-4.7, behind
``torch.autograd.Function``:

* forward  -- sequential time stepping (Alg. 1 applied Nt times) that keeps only the slice
              boundary states u_s = (T_{Ms}, theta_{Ms}), s = 0..N_tau (checkpoints), not the
              history: ``ptg_fine_propagate_slices`` in chained mode with no history window.
* backward -- for s = N_tau-1 .. 0: recompute slice s's history T_{Ms..M(s+1)} from its
              checkpoint into an (M+1)-row window (``ptg_fine_propagate_slices`` on one slice),
              then run the adjoint kernel over that slice from v_{s+1} (``ptg_adjoint_sweep``
              on one slice with the window), which yields v_s = (lambda_{Ms+1}, g_{Ms+1}).
              The gradient is g_1, scaled by the incoming gradient of Theta.

Device memory: (N_tau + 1) N_n for the checkpoints plus (M + 1) N_n for the window, instead
of (N_t + 1) N_n for the full history.  Every step runs in the library's CUDA kernels; the
recomputed history is bit-identical to the forward's because the kernels are deterministic.
"""
from __future__ import annotations

import torch

from .api import Operator
from ._ffi import PTG_SLICES_CHAINED, PTG_SLICES_PARALLEL


class _Checkpoints:
    def __init__(self, op: Operator):
        z = op.zeros
        self.U_T, self.U_th = z(op.Ntau + 1, op.Nn), z(op.Ntau + 1)
        self.window = z(op.M + 1, op.Nn)
        self.F_T, self.F_th = z(op.Ntau, op.Nn), z(op.Ntau)
        self.V_l, self.V_g = z(op.Ntau + 1, op.Nn), z(op.Ntau + 1, op.Ne)


def forward_checkpointed(op: Operator, rho: torch.Tensor, T0: torch.Tensor | None = None) -> tuple[torch.Tensor, _Checkpoints]:
    """Sequential primal pass keeping only the slice-boundary states; returns (Theta, ckpt)."""
    ck = _Checkpoints(op)
    op.assemble(rho.detach().contiguous())
    if T0 is not None:
        ck.U_T[0].copy_(T0)
    op.fine_propagate_slices(ck.U_T, ck.U_th, ck.U_T[1:], ck.U_th[1:], T_hist=None, schedule=PTG_SLICES_CHAINED)
    return ck.U_th[op.Ntau].clone(), ck


def backward_checkpointed(op: Operator, ck: _Checkpoints) -> torch.Tensor:
    """Reverse sweep over the slices with per-slice recomputation; returns dTheta/drho [Ne].
    Requires that the op still holds the design of the forward pass."""
    M, Ntau = op.M, op.Ntau
    Theta = ck.U_th[Ntau:Ntau + 1]
    ck.V_l[Ntau].zero_()
    ck.V_g[Ntau].zero_()
    for s in range(Ntau - 1, -1, -1):
        # recompute T_{Ms+1..M(s+1)} into window rows 1..M from the checkpoint u_s (row 0 = T_{Ms})
        ck.window[0].copy_(ck.U_T[s])
        op.fine_propagate_slices(ck.U_T, ck.U_th, ck.F_T, ck.F_th, T_hist=ck.window, hist_j0=M * s,
                                 schedule=PTG_SLICES_PARALLEL, s0=s, ns=1)
        op.adjoint_sweep(ck.window, Theta, ck.V_l, ck.V_g, ck.V_l, ck.V_g, hist_j0=M * s,
                         schedule=PTG_SLICES_PARALLEL, s0=s, ns=1)
    return ck.V_g[0].clone()


class ParaTopoFn(torch.autograd.Function):
    """Theta = ParaTopoFn.apply(rho, op): the power-mean temperature objective of the design rho
    (FP64 CUDA tensor [Ne]) for the problem held by the ``Operator`` op; differentiable in rho."""

    @staticmethod
    def forward(ctx, rho: torch.Tensor, op: Operator):
        Theta, ck = forward_checkpointed(op, rho)
        ctx.op = op
        ctx.ck = ck
        return Theta

    @staticmethod
    def backward(ctx, grad_out):
        g = backward_checkpointed(ctx.op, ctx.ck)
        return grad_out * g, None


def objective(rho: torch.Tensor, op: Operator) -> torch.Tensor:
    """Differentiable Theta(rho) (see ``ParaTopoFn``)."""
    return ParaTopoFn.apply(rho, op)
