"""The one-shot pass with its slices split over several processes (one GPU each).

The parallel parts of a Parareal iteration are independent over slices (Sec. 4.2, Fig. 2: each
slice's F and G depend only on that slice's start state), and the sequential correction sweep
(Eq. 4.9 forward, Eq. 4.14 reverse) needs every slice's F and G results.  So each rank takes a
contiguous range of slices, propagates them, and the ranks exchange the slice results once per
direction; every rank then runs the identical sequential sweep on identical inputs, which
needs no broadcast afterwards because the library's kernels are deterministic.

Per rank, with slices s0 .. s0 + ns - 1:
  1. F_pri and G_pri of its slices (ptg_fine_propagate_slices, ptg_coarse_sweep_slices); the
     history rows of its slices are written locally.
  2. All-gather of F(u_s^old) = (F_T, F_theta) and G(u_s^old) = (G_T, G_theta) of every slice, and of
     the first history row T_{Ms+1} of every slice (the coarse adjoint of slice s reads T_{Ms+1}
     and T_{M(s-1)+1}, the latter on the previous rank).
  3. The forward correction sweep on every rank: u^new, the corrected rows T_{M(s+1)}, Theta.
  4. F_adj and G_adj of its slices (they read only the rows of their own slices, the corrected
     coarse rows and the gathered first rows).
  5. All-gather of (F_lam, F_g) and (G_lam, G_g) of every slice.
  6. The reverse correction sweep on every rank: v^new and the gradient g_1.

Only the slices' own history rows, the corrected coarse rows and the first rows are valid on a
rank; the rest of its history buffer is not written.  Every step runs in the library's kernels;
this module only orders the calls and moves rows between processes through
torch.distributed (NCCL for CUDA tensors, or host staging for a CPU backend such as gloo).

The propagation calls go through an ``op`` object with the methods of ``api.Operator``
(fine_propagate_slices, coarse_sweep_slices, parareal_correct, adjoint_sweep) and the sizes
Nt, Ntau, M, Nn, Ne; buffers have the shapes of ``api.PassBuffers``.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from ._ffi import PTG_ADJOINT, PTG_PRIMAL


def slice_range(Ntau: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous balanced partition of the Ntau slices: (s0, ns) of `rank`; the first
    Ntau mod world ranks take one slice more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("invalid rank / world size")
    base, extra = divmod(Ntau, world)
    ns = base + (1 if rank < extra else 0)
    s0 = rank * base + min(rank, extra)
    return s0, ns


def _all_gather_rows(parts: list[torch.Tensor], Ntau: int, world: int, group=None):
    """Row-block all-gather: every tensor in `parts` has Ntau rows (slice-indexed); on entry each
    rank holds valid rows for its own slices, on return every rank holds all rows.  Blocks are
    padded to the largest share so that every rank sends the same byte count; CUDA tensors on
    a backend without CUDA collectives are staged through host memory."""
    nsmax = -(-Ntau // world)
    backend = dist.get_backend(group)
    me = dist.get_rank(group)
    s0, ns = slice_range(Ntau, world, me)
    for t in parts:
        flat = t.reshape(Ntau, -1)
        where = "cpu" if (t.is_cuda and backend != "nccl") else flat.device
        send = torch.zeros((nsmax, flat.shape[1]), dtype=flat.dtype, device=where)
        send[:ns].copy_(flat[s0:s0 + ns])
        recv = [torch.empty_like(send) for _ in range(world)]
        dist.all_gather(recv, send, group=group)
        for r in range(world):
            a, n = slice_range(Ntau, world, r)
            if r != me and n:
                flat[a:a + n].copy_(recv[r][:n])


def sharded_oneshot_pass(op, buf, world: int | None = None, rank: int | None = None, group=None, stream=None):
    """The iteration body of Alg. 3 (as ``api.oneshot_pass``) with this rank's share of the
    slices; returns (Theta, grad) views, identical on every rank.  buf.U_* / buf.V_* hold the
    warm start on every rank; on return buf.U_*_new / buf.V_*_new hold the corrected states."""
    world = dist.get_world_size(group) if world is None else world
    rank = dist.get_rank(group) if rank is None else rank
    Ntau, M = op.Ntau, op.M
    s0, ns = slice_range(Ntau, world, rank)
    first_rows = buf.T_hist[1::M][:Ntau]          # T_{Ms+1}, s = 0..Ntau-1 (a strided view)
    first = torch.zeros((Ntau,) + tuple(buf.T_hist.shape[1:]), dtype=buf.T_hist.dtype, device=buf.T_hist.device)
    # primal: F and G of this rank's slices, exchange, then the sequential sweep everywhere
    if ns:
        op.fine_propagate_slices(buf.U_T, buf.U_th, buf.F_T, buf.F_th, T_hist=buf.T_hist, s0=s0, ns=ns, stream=stream)
        op.coarse_sweep_slices(PTG_PRIMAL, s0, ns, buf.U_T, buf.U_th, buf.G_T, buf.G_th, stream=stream)
        first[s0:s0 + ns].copy_(first_rows[s0:s0 + ns])
    _sync(buf.T_hist, stream)
    _all_gather_rows([buf.F_T, buf.F_th, buf.G_T, buf.G_th, first], Ntau, world, group)
    first_rows.copy_(first)
    buf.U_T_new[0].copy_(buf.U_T[0])
    buf.U_th_new[0].copy_(buf.U_th[0])
    op.parareal_correct(PTG_PRIMAL, buf.F_T, buf.F_th, buf.G_T, buf.G_th, buf.U_T_new, buf.U_th_new,
                        T_hist=buf.T_hist, stream=stream)
    Theta = buf.U_th_new[Ntau:Ntau + 1]
    # adjoint: F and G of this rank's slices, exchange, then the reverse sweep everywhere
    if ns:
        op.adjoint_sweep(buf.T_hist, Theta, buf.V_l, buf.V_g, buf.F_l, buf.F_g, s0=s0, ns=ns, stream=stream)
        op.coarse_sweep_slices(PTG_ADJOINT, s0, ns, buf.V_l, buf.V_g, buf.G_l, buf.G_g, T_hist=buf.T_hist,
                               Theta=Theta, stream=stream)
    _sync(buf.T_hist, stream)
    _all_gather_rows([buf.F_l, buf.F_g, buf.G_l, buf.G_g], Ntau, world, group)
    op.parareal_correct(PTG_ADJOINT, buf.F_l, buf.F_g, buf.G_l, buf.G_g, buf.V_l_new, buf.V_g_new,
                        T_hist=buf.T_hist, Theta=Theta, stream=stream)
    return Theta, buf.V_g_new[0]


def _sync(t: torch.Tensor, stream):
    """Collectives run on torch's current stream: make the library's stream (if another) finish first."""
    if t.is_cuda:
        if stream is not None and stream != torch.cuda.current_stream(t.device):
            stream.synchronize()
