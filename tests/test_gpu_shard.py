"""The slice-sharded one-shot pass with the CUDA library: two processes on cuda:0, each
propagating half of the slices, exchanging the slice results through gloo (host staging), and
running the correction sweeps redundantly.  No kernel waits on another process's kernels: the
only exchange is on the host between launches.  With the launch geometry of every slice kind
fixed to that of the single-process pass, each rank's result must equal the single-process
pass bit for bit, and the oracle within the parity tolerances."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu


def _worker(rank, world, port, precision, q):
    import workloads as W
    from oracle import Operator as OracleOp, coarse_states_from_sequential, oneshot_pass as o_oneshot
    from paper_2411_19030_gb300 import PassBuffers, oneshot_pass
    from paper_2411_19030_gb300.shard import sharded_oneshot_pass, slice_range
    from tests.gpu_helpers import FP64_TOL, MIXED_G_TOL, MIXED_T_TOL, dev, gpu_operator, host, rel_err
    from tests.problems import make_problem

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Nt, Ntau = 30, 6
        prob = make_problem(26, 19, Nt=Nt, Ntau=Ntau, dt=0.6 / Nt, material="table1", sink="left_wide",
                            q_time=W.q_time_paper(Nt, 0.6 / Nt))
        rho = W.rho_uniform(26, 19, 51, 0.05, 0.95)
        rho_old = W.rho_warm_perturb(rho, seed=52, amp=0.05)
        U_old, V_old, _ = coarse_states_from_sequential(OracleOp(prob, rho_old))
        ref = o_oneshot(OracleOp(prob, rho), U_old, V_old)
        op = gpu_operator(prob, precision, rtol=1e-13 if precision == "fp64" else 1e-10)
        for kind in (0, 1, 3, 4):                     # the single-process launch geometry
            pl = op.plan(kind, Ntau)
            op.set_plan(kind, pl["cs"], pl["ng"])
        bufs = []
        for _ in range(2):
            b = PassBuffers(op)
            b.U_T.copy_(dev(U_old[0])); b.U_th.copy_(dev(U_old[1]))
            b.V_l.copy_(dev(V_old[0])); b.V_g.copy_(dev(V_old[1]))
            bufs.append(b)
        op.assemble(dev(rho))
        # single process, every slice, with the adjoint coarse propagators solved directly as the
        # sharded pass does (not as the two overlapped parts)
        Th1, g1 = oneshot_pass(op, bufs[0], overlap=False)
        Th2, g2 = sharded_oneshot_pass(op, bufs[1])              # this rank's slices + exchange
        torch.cuda.synchronize()
        s0, ns = slice_range(Ntau, world, rank)
        M = prob.M
        rows = sorted(set(range(M * s0 + 1, M * (s0 + ns) + 1)) | set(range(0, Nt + 1, M)) | set(range(1, Nt + 1, M)))
        a, b = bufs
        same = {
            "U_new": torch.equal(a.U_T_new, b.U_T_new), "theta_new": torch.equal(a.U_th_new, b.U_th_new),
            "T_hist rows": torch.equal(a.T_hist[rows], b.T_hist[rows]),
            "V_new": torch.equal(a.V_l_new, b.V_l_new), "g_new": torch.equal(a.V_g_new, b.V_g_new),
            "grad": torch.equal(g1, g2), "Theta": torch.equal(Th1, Th2),
        }
        tol_t, tol_g = (FP64_TOL, FP64_TOL) if precision == "fp64" else (MIXED_T_TOL, MIXED_G_TOL)
        errs = {"T_hist": (rel_err(host(b.T_hist)[rows], ref["T_hist"][rows]), tol_t),
                "Theta": (rel_err(host(Th2), [ref["Theta"]]), tol_t),
                "V_new": (rel_err(host(b.V_l_new), ref["V"][0]), tol_g),
                "grad": (rel_err(host(g2), ref["grad"]), tol_g)}
        q.put((rank, ns, same, errs, op.stats()["status"]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_sharded_pass_two_processes_matches_single_process_and_oracle(precision):
    from tests.gpu_helpers import ensure_built
    ensure_built()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, precision, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(ns for _, ns, *_ in results) == [3, 3]
    for rank, ns, same, errs, status in results:
        assert status == 0
        bad = [k for k, ok in same.items() if not ok]
        assert not bad, f"rank {rank}: differs from the single-process pass in {bad}"
        for k, (e, tol) in errs.items():
            assert e <= tol, f"rank {rank}: {k} error {e:.3e} > {tol:.1e}"
