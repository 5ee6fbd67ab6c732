"""The slice-sharded one-shot pass (paper_2411_19030_gb300.shard) on CPU processes over gloo.

Each rank propagates a contiguous range of slices, the ranks all-gather the slice results and
the first history row of every slice, and every rank runs the identical correction sweeps.
Here the library calls are stood in for by the oracle's propagators (F_pri, G_pri, F_adj, G_adj
of Sec. 4.4 and the sweeps of Eq. 4.9 / 4.14) acting on CPU tensors, so the test checks the
partition, the exchange and the order of the calls: on every rank the result must equal the
oracle's single-process one-shot pass bit for bit (same arithmetic on the same inputs).  The
same driver with the CUDA library is checked on the GPU in tests/test_gpu_shard.py."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from oracle import Operator as OracleOp, coarse_states_from_sequential, oneshot_pass as o_oneshot
from oracle.parareal import F_adj, F_pri, G_adj, G_pri
from paper_2411_19030_gb300._ffi import PTG_PRIMAL
from paper_2411_19030_gb300.shard import sharded_oneshot_pass, slice_range
from tests.problems import make_problem


class OracleSliceOp:
    """The four propagation calls of the library's op on CPU tensors, computed by the oracle."""

    def __init__(self, op: OracleOp):
        self.o = op
        p = op.prob
        self.Nt, self.Ntau, self.M, self.Nn, self.Ne = p.Nt, p.Ntau, p.M, p.Nn, p.Ne

    def fine_propagate_slices(self, U_T, U_th, F_T, F_th, T_hist=None, s0=0, ns=None, stream=None):
        for s in range(s0, s0 + ns):
            T, th, inter = F_pri(self.o, s, U_T[s].numpy(), float(U_th[s]))
            F_T[s] = torch.from_numpy(T)
            F_th[s] = th
            T_hist[self.M * s + 1:self.M * (s + 1) + 1] = torch.from_numpy(inter)

    def coarse_sweep_slices(self, direction, s0, ns, X_field, X_aux, G_field, G_aux, T_hist=None, Theta=None,
                            stream=None):
        for s in range(s0, s0 + ns):
            if direction == PTG_PRIMAL:
                T, th = G_pri(self.o, s, X_field[s].numpy(), float(X_aux[s]))
                G_field[s], G_aux[s] = torch.from_numpy(T), th
            else:
                lam, g = G_adj(self.o, s, X_field[s + 1].numpy(), X_aux[s + 1].numpy(), T_hist.numpy(), float(Theta))
                G_field[s], G_aux[s] = torch.from_numpy(lam), torch.from_numpy(g)

    def adjoint_sweep(self, T_hist, Theta, V_lam, V_g, F_lam, F_g, s0=0, ns=None, stream=None):
        for s in range(s0, s0 + ns):
            lam, g = F_adj(self.o, s, V_lam[s + 1].numpy(), V_g[s + 1].numpy(), T_hist.numpy(), float(Theta))
            F_lam[s], F_g[s] = torch.from_numpy(lam), torch.from_numpy(g)

    def parareal_correct(self, direction, F_field, F_aux, G_field, G_aux, X_field, X_aux, T_hist=None, Theta=None,
                         stream=None):
        M, Ntau = self.M, self.Ntau
        if direction == PTG_PRIMAL:
            T_hist[0] = X_field[0]
            for s in range(Ntau):
                gT, gth = G_pri(self.o, s, X_field[s].numpy(), float(X_aux[s]))
                X_field[s + 1] = torch.from_numpy(gT) + F_field[s] - G_field[s]
                X_aux[s + 1] = gth + F_aux[s] - G_aux[s]
                T_hist[M * (s + 1)] = X_field[s + 1]
        else:
            X_field[Ntau] = 0.0
            X_aux[Ntau] = 0.0
            for s in range(Ntau - 1, -1, -1):
                gl, gg = G_adj(self.o, s, X_field[s + 1].numpy(), X_aux[s + 1].numpy(), T_hist.numpy(), float(Theta))
                X_field[s] = torch.from_numpy(gl) + F_field[s] - G_field[s]
                X_aux[s] = torch.from_numpy(gg) + F_aux[s] - G_aux[s]


class Buffers:
    def __init__(self, prob):
        Nt, Ntau, Nn, Ne = prob.Nt, prob.Ntau, prob.Nn, prob.Ne
        z = lambda *s: torch.zeros(*s, dtype=torch.float64)
        self.T_hist = z(Nt + 1, Nn)
        self.F_T, self.F_th, self.G_T, self.G_th = z(Ntau, Nn), z(Ntau), z(Ntau, Nn), z(Ntau)
        self.F_l, self.F_g, self.G_l, self.G_g = z(Ntau, Nn), z(Ntau, Ne), z(Ntau, Nn), z(Ntau, Ne)
        self.U_T, self.U_th, self.V_l, self.V_g = z(Ntau + 1, Nn), z(Ntau + 1), z(Ntau + 1, Nn), z(Ntau + 1, Ne)
        self.U_T_new, self.U_th_new = z(Ntau + 1, Nn), z(Ntau + 1)
        self.V_l_new, self.V_g_new = z(Ntau + 1, Nn), z(Ntau + 1, Ne)


def _case(Ntau):
    prob = make_problem(7, 5, Nt=3 * Ntau, Ntau=Ntau, dt=0.5 / (3 * Ntau), material="table1", sink="left_wide",
                        q_time=W.q_time_paper(3 * Ntau, 0.5 / (3 * Ntau)))
    rho = W.rho_uniform(7, 5, 31, 0.1, 0.9)
    rho_old = W.rho_warm_perturb(rho, seed=32, amp=0.05)
    return prob, rho, rho_old


def _worker(rank, world, port, Ntau, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob, rho, rho_old = _case(Ntau)
        U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
        ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
        op = OracleSliceOp(OracleOp(prob, rho))
        buf = Buffers(prob)
        buf.U_T.copy_(torch.from_numpy(U_old[0])); buf.U_th.copy_(torch.from_numpy(U_old[1]))
        buf.V_l.copy_(torch.from_numpy(V_old[0])); buf.V_g.copy_(torch.from_numpy(V_old[1]))
        Theta, grad = sharded_oneshot_pass(op, buf)
        s0, ns = slice_range(Ntau, world, rank)
        M = prob.M
        rows = sorted(set(range(M * s0 + 1, M * (s0 + ns) + 1)) | set(range(0, prob.Nt + 1, M))
                      | set(range(1, prob.Nt + 1, M)))
        checks = {
            "U_new": np.array_equal(buf.U_T_new.numpy(), ref["U"][0]),
            "theta_new": np.array_equal(buf.U_th_new.numpy(), ref["U"][1]),
            "Theta": float(Theta) == ref["Theta"],
            "T_hist rows": np.array_equal(buf.T_hist.numpy()[rows], ref["T_hist"][rows]),
            "V_new": np.array_equal(buf.V_l_new.numpy(), ref["V"][0]),
            "g_new": np.array_equal(buf.V_g_new.numpy(), ref["V"][1]),
            "grad": np.array_equal(grad.numpy(), ref["grad"]),
        }
        q.put((rank, ns, checks))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,Ntau", [(2, 4), (2, 5), (3, 4)])
def test_sharded_pass_equals_single_process_oracle_pass(world, Ntau):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, Ntau, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sum(ns for _, ns, _ in results) == Ntau
    for rank, ns, checks in results:
        bad = [k for k, ok in checks.items() if not ok]
        assert not bad, f"rank {rank}: {bad}"


def test_slice_range_partitions_contiguously():
    for Ntau in (1, 4, 5, 32, 33):
        for world in (1, 2, 3, 8):
            got = [slice_range(Ntau, world, r) for r in range(world)]
            s = 0
            for s0, ns in got:
                assert s0 == s and ns >= 0
                s += ns
            assert s == Ntau
            assert max(n for _, n in got) - min(n for _, n in got) <= 1


def _failing_worker(rank, world, port, q):
    """Rank 1's fine propagation raises (a host-side injected failure) before the first exchange;
    rank 1 then leaves.  Rank 0 must learn of it from its next collective, which ends with an error
    within the process group's timeout instead of waiting for ever."""
    import datetime
    import time

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    prob, rho, rho_old = _case(4)
    U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
    op = OracleSliceOp(OracleOp(prob, rho))
    buf = Buffers(prob)
    buf.U_T.copy_(torch.from_numpy(U_old[0])); buf.U_th.copy_(torch.from_numpy(U_old[1]))
    buf.V_l.copy_(torch.from_numpy(V_old[0])); buf.V_g.copy_(torch.from_numpy(V_old[1]))
    if rank == 1:
        def fail(*args, **kwargs):
            raise RuntimeError("injected failure of the fine propagation")
        op.fine_propagate_slices = fail
    t0 = time.monotonic()
    try:
        sharded_oneshot_pass(op, buf)
        q.put((rank, "finished", "", time.monotonic() - t0))
    except Exception as e:                                  # noqa: BLE001 -- reported to the test
        q.put((rank, "error", f"{type(e).__name__}: {str(e)[:120]}", time.monotonic() - t0))
    q.close()
    q.join_thread()
    os._exit(0)                                             # leave without a closing collective


def test_a_failing_rank_ends_the_others_collectives_with_an_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        results = {r: (status, msg, secs) for r, status, msg, secs in (q.get(timeout=120) for _ in range(2))}
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert results[1][0] == "error" and "injected failure" in results[1][1]
    assert results[0][0] == "error", results[0]             # rank 0's all-gather did not complete
    assert results[0][2] < 60.0                             # bounded by the process group's timeout
