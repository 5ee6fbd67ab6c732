"""The design map on the device (density filter, projection, area fraction, chain rule) and
the one-shot design loop of Alg. 3 (GPU pass + host MMA) against the oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import workloads as W
from oracle.design import Design, design_loop
from paper_2411_19030_gb300.design import DesignMap, OneShotLoop
from tests.gpu_helpers import assert_close, dev, ensure_built, gpu_operator, host
from tests.problems import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("nx,ny,r_fil,beta", [(64, 48, 0.07, 32.0), (13, 9, 0.25, 4.0), (30, 30, 0.01, 8.0)])
def test_design_map_matches_oracle(nx, ny, r_fil, beta):
    h = 1.0 / max(nx, ny)
    ref = Design(nx, ny, h, r_fil, beta, 0.5)
    chi = W.rho_uniform(nx, ny, 17, 0.0, 1.0)
    y = W.rho_uniform(nx, ny, 18, -1.0, 1.0)
    rho_r, dp_r = ref.forward(chi)
    dm = DesignMap(nx, ny, h, r_fil, beta, 0.5)
    rho, dp, g, gv, vol = (torch.empty(nx * ny, dtype=torch.float64, device="cuda") for _ in range(5))
    dm.forward(dev(chi), rho, dp)
    dm.backward(dp, dev(y), g)
    dm.backward(dp, None, gv)
    dm.volume(rho, vol)
    torch.cuda.synchronize()
    assert_close("rho", host(rho), rho_r, 1e-13)
    assert_close("dproj", host(dp), dp_r, 1e-13)
    assert_close("H^T", host(g), ref.backward(dp_r, y), 1e-13)
    assert_close("volume gradient", host(gv), ref.volume_gradient(dp_r), 1e-13)
    assert abs(float(vol[0].item()) - float(np.mean(rho_r))) < 1e-14


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32_refine", 1e-5)])
def test_design_loop_matches_oracle(precision, tol):
    """Five iterations of Alg. 3 (one sequential, four one-shot) with MMA: the objective, the
    area fraction and the design of every iteration."""
    Nt = 32
    prob = make_problem(20, 16, Nt=Nt, Ntau=4, dt=1.0 / Nt, material="table1", sink="bottom", p=8.0,
                        q_time=W.q_time_paper(Nt, 1.0 / Nt))
    r_fil, beta, a_max, iters = 0.12, 8.0, 0.3, 5
    chi0 = np.full(prob.Ne, a_max)
    ref = design_loop(prob, r_fil, beta, 0.5, a_max, chi0, iters)
    op = gpu_operator(prob, precision, rtol=1e-13 if precision == "fp64" else 1e-10)
    loop = OneShotLoop(op, DesignMap(prob.nx, prob.ny, prob.h, r_fil, beta, 0.5), a_max)
    chi = chi0.copy()
    for k in range(iters):
        out = loop.iterate(chi, first=(k == 0))
        chi = out["chi"]
        assert abs(out["Theta"] - ref["Theta"][k]) <= tol * abs(ref["Theta"][k]), k
        assert abs(out["volume"] - ref["volume"][k]) <= tol, k
        assert np.max(np.abs(chi - ref["chi"][k])) <= 10 * tol, k
    assert op.stats()["status"] == 0


def test_design_loop_resumes_from_a_saved_state(tmp_path):
    """A loop saved after two design iterations and resumed in fresh objects (a new operator,
    buffers and MMA) continues exactly as the uninterrupted loop: the state it carries is the
    design chi, the warm-start coarse states u^old and v^old, Theta_1 and the MMA history."""
    Nt = 32
    prob = make_problem(20, 16, Nt=Nt, Ntau=4, dt=1.0 / Nt, material="table1", sink="bottom", p=8.0,
                        q_time=W.q_time_paper(Nt, 1.0 / Nt))
    r_fil, beta, a_max = 0.12, 8.0, 0.3
    chi0 = np.full(prob.Ne, a_max)

    def new_loop():
        op = gpu_operator(prob, "fp32_refine", rtol=1e-10)
        return OneShotLoop(op, DesignMap(prob.nx, prob.ny, prob.h, r_fil, beta, 0.5), a_max)

    full = new_loop().run(chi0, 5)
    first = new_loop().run(chi0, 2)
    saver = new_loop()
    saver.run(chi0, 2)
    path = str(tmp_path / "loop_state.npz")
    saver.save(path, first["chi"], 2)
    resumed = new_loop()
    chi, done = resumed.load(path)
    assert done == 2 and np.array_equal(chi, first["chi"])
    rest = resumed.run(chi, 5, start=done)
    assert rest["Theta"] == full["Theta"][2:]
    assert rest["volume"] == full["volume"][2:]
    assert np.array_equal(rest["chi"], full["chi"])
    with pytest.raises(ValueError):
        op2 = gpu_operator(make_problem(12, 10, Nt=Nt, Ntau=4, dt=1.0 / Nt), "fp32_refine")
        OneShotLoop(op2, DesignMap(12, 10, 1 / 12, r_fil, beta, 0.5), a_max).load(path)
